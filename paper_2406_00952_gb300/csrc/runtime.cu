// Host runtime and C ABI (include/pcb.h): problem creation (validation, spectral and twiddle
// tables of Sec. 3.5, launch shapes), workspaces, and the batched solver loops (MINRES,
// FGMRES with CGS2, FP64 iterative refinement around an FP32 preconditioner).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "pcb_internal.cuh"

namespace pcb {
// launchers defined in the other translation units
cudaError_t launch_precond_fast(const Batch& B, int kind, int prec, int in_slot, int out_slot);
cudaError_t launch_precond_mg(const Batch& B, const Geom& g, int kind, int prec, int cycles, int in_slot,
                              int out_slot);
void mg_release(const void* ws);
long long mg_launch_total();
cudaError_t launch_matvec(const Batch& B, int op, int x_slot, int out_slot, int aux_slot, int epi);
cudaError_t launch_rhs(const Geom& g, cudaStream_t st, int op, const double* gs, const double* fs, const double* y0,
                       double* b);
cudaError_t launch_recover(const Geom& g, cudaStream_t st, const double* x, double* y, double* p);
cudaError_t launch_copy_mapped(cudaStream_t st, const double* src, double* dst, long long n);
cudaError_t launch_fem_spatial(const Batch& B, int mode, int op, int in_slot, int out_slot);

// device address of page-locked host memory the device maps, or null (pageable memory)
static const void* mapped_ptr(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// n doubles between a host buffer and device memory: the copy kernel when the host side is
// page-locked and mapped, cudaMemcpyAsync otherwise.  *kernels counts the copy kernels launched.
static cudaError_t copy_host(double* dst, const double* src, size_t n, bool to_device, cudaStream_t st,
                             long long* kernels) {
  const void* map = mapped_ptr(to_device ? (const void*)src : (const void*)dst);
  if (map) {
    if (kernels) ++*kernels;
    return to_device ? launch_copy_mapped(st, (const double*)map, dst, (long long)n)
                     : launch_copy_mapped(st, src, (double*)map, (long long)n);
  }
  return cudaMemcpyAsync(dst, src, n * sizeof(double), to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost,
                         st);
}
cudaError_t launch_dot(const Batch& B, int sa, int sb);
cudaError_t launch_reduce(const Batch& B, const int* off, int nper, int which, int step, double tol, int j,
                          int restart);
cudaError_t launch_axpby(const Batch& B, int mode, int sx, int sy, int sz);
cudaError_t launch_minres_wx(const Batch& B, int sy, int sw, int sw2, int sx);
// j < 0: each instance at its own Arnoldi index (from Scal), all of them <= jmax when jmax >= 0
cudaError_t launch_multidot(const Batch& B, int svbase, int j, int sw, int jmax = -1);
cudaError_t launch_reduce_multi(const Batch& B, int j, int pass);
cudaError_t launch_multiaxpy(const Batch& B, int svbase, int j, int sw, int pass, int jmax = -1);
cudaError_t launch_swap(const Batch& B, int a0, int b0, int a1, int b1, int a2, int b2);
cudaError_t launch_setslot(const Batch& B, int dst, int base, int k, int per_j = 0);
size_t mg_workspace_bytes(const Geom& g);
void matvec_shape(Geom& g);
bool mg_available();
int dst_Q(int N);
int time_Q(int n);
bool q_supported(int Q);
size_t dst_smem_bytes(const Geom& g, int p);
size_t time_smem_bytes(const Geom& g, int p);
int padded_len_host(int len);
int pipe_dst_p(const Geom& g);
int pipe_time_p(const Geom& g);
int pipe_dst_code(const Geom& g);
int pipe_time_code(const Geom& g);
int pipe_time_cols(int n, int zeta_pi);
int pipe_dst_lines(int L);
cudaError_t upload_constants();
struct TableLayout { size_t kap, mud, muf, twdd, twdf, twtd, twtf, pred, pref, ax, ay, dg, ms, bytes; };
cudaError_t mg_setup(Geom& g, void* ws, const double* a_edges_host, double a0);

// step ids of the scalar kernels (mirror krylov.cu)
enum { SS_NONE = 0, SS_MINRES_INIT, SS_MINRES_ALFA, SS_MINRES_GIVENS, SS_NORM, SS_GMRES_ARNOLDI, SS_GMRES_START,
       SS_BNORM };
enum { AX_COPY = 0, AX_MINRES_R = 1, AX_SCALE_INV_BETA = 2, AX_SCALE_INV_HNORM = 3, AX_ADD = 4, AX_ZERO = 5 };
enum { EPI_PLAIN = 0, EPI_RESID = 1, EPI_MINRES = 2 };
constexpr int EPI_FAST = 8;     // the inner MINRES product of a mixed-precision solve (matvec.cu)
enum { PK_ABS_PS = 1, PK_PS = 2, PK_PMS = 3 };

// vector slots
enum {
  SL_UIN = 0, SL_UOUT = 1,           // user buffers of standalone calls
  SL_X = 2, SL_B = 3,                // solve: solution and right-hand side (outer)
  SL_XI = 4, SL_BI = 5,              // inner solve solution / right-hand side
  SL_R1 = 6, SL_R2 = 7, SL_Y = 8, SL_YO = 9, SL_Q = 10, SL_W = 11, SL_W2 = 12,
  SL_R = 13, SL_VBASE = 14, SL_ZBASE = 15, SL_VJ = 16, SL_ZJ = 17, SL_VJ1 = 18,
  SL_UAUX = 19                       // third user buffer of standalone calls
};

}  // namespace pcb

using namespace pcb;

struct pcb_problem {
  pcb_desc desc;
  Geom g;                 // host mirror (device pointers inside)
  cudaStream_t stream;
  int device;
  // device allocations
  void* tables = nullptr;
  void* scratch = nullptr;
  void* mgws = nullptr;
  double* vec_minres = nullptr;   // 7 vectors
  double* vec_mixed = nullptr;    // 2 vectors (inner rhs / solution)
  double* vec_gmres = nullptr;    // R + V(restart+1) + Z(restart)
  int gmres_restart = 0;
  long long bytes = 0;
  // single-instance batch
  Geom* dG = nullptr;
  Slots hS;
  Slots* dS = nullptr;
  Scal* dSc = nullptr;
  int* doff = nullptr;            // 12 offset arrays of length 2
  double* partial = nullptr;
  Scal* hSc = nullptr;            // pinned host copy
  Slots* hSpin = nullptr;         // pinned staging for slot uploads
  Batch B;
  double* host_io = nullptr;      // device staging for pcb_solve_host (b, x)
  // CUDA graph of one MINRES iteration (captured on a private stream, replayed on `stream`)
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t git = nullptr;
  int git_kind = -1, git_prec = -1, git_sx = -1;
  long long git_launches = 0;
  // CUDA graphs of the FGMRES Arnoldi steps, one per index j, for one (preconditioner, precision,
  // restart) setting
  cudaGraphExec_t garn[PCB_MAX_RESTART] = {};
  long long garn_launches[PCB_MAX_RESTART] = {};
  int garn_kind = -1, garn_prec = -1, garn_restart = -1;
  double* dtol = nullptr;         // device copy of the running tolerance read by the scalar steps
  // per-solve counters and optional event profiling
  long long launches = 0;
  int prec_applies = 0, matvecs = 0, matvecs_inner = 0;
  bool prof = false;
  std::vector<cudaEvent_t> ev_prec, ev_mv, ev_mvi;   // pairs (start, stop); ev_mvi: two-word products
  int ev_prec_used = 0, ev_mv_used = 0, ev_mvi_used = 0;
};

namespace {

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

int cuda_status(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return PCB_ERR_OUT_OF_MEMORY; }
  return PCB_ERR_CUDA;
}

bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

bool make_plan(int M, FftPlan& p) {
  p.M = M;
  p.nst = 0;
  int r = M;
  // prefer radix 8, then 4, finish with 2 and 3
  while (r % 3 == 0) { if (p.nst >= PCB_MAX_STAGES) return false; p.rad[p.nst++] = 3; r /= 3; }
  while (r % 8 == 0) { if (p.nst >= PCB_MAX_STAGES) return false; p.rad[p.nst++] = 8; r /= 8; }
  while (r % 4 == 0) { if (p.nst >= PCB_MAX_STAGES) return false; p.rad[p.nst++] = 4; r /= 4; }
  while (r % 2 == 0) { if (p.nst >= PCB_MAX_STAGES) return false; p.rad[p.nst++] = 2; r /= 2; }
  return r == 1;
}

int vec_blocks_for(long long len) {
  long long b = (len + 2047) / 2048;
  if (b > 2432) b = 2432;
  if (b < 1) b = 1;
  return (int)b;
}

int pow2_floor(int v) { int p = 1; while (p * 2 <= v) p *= 2; return p; }

void set_shapes(Geom& g) {
  const int pd = pipe_dst_p(g), pt = pipe_time_p(g);   // pipelined FP32 passes: 256/P lines a tile
  g.lr = pd ? g.L + 16 : g.N;      // + 16: rows stay 64-byte aligned, stride off a power of two
  g.mp = (long long)g.N * g.lr;
  const int lsd = padded_len_host(g.L), lst = padded_len_host(g.n);
  const int Pd = 2 * g.L / g.dst_q, Pt = g.n / g.time_q;
  const int lpwd = 32 / Pd, lpwt = 32 / Pt;
  // complex elements per tile: FP64, FP32 (~68 KB); the autotuner may halve or double them
  const int bs = tune_budget_shift(g.tune);
  const int budget[2] = {bs == 1 ? 2150 : bs == 2 ? 8600 : 4300, bs == 1 ? 4300 : bs == 2 ? 17200 : 8600};
  for (int p = 0; p < 2; ++p) {
    // powers of two (the kernels split thread indices with shifts) that are multiples of lpw
    // Q = 32 lines use one warp each plus a per-warp transpose scratch: 8 lines per block
    int lpb = g.dst_q == 32 ? 8 : std::max(lpwd, pow2_floor(std::min(256, std::max(1, budget[p] / lsd))));
    if (p == 1 && pd) lpb = pipe_dst_lines(g.L);
    g.dst_lpb[p] = lpb;
    int lpbj = std::max(lpwd, std::min(lpb, pow2_floor(std::max(1, g.N))));
    if (p == 1 && pd) lpbj = pipe_dst_lines(g.L);
    g.dst_lpb_j[p] = lpbj;
    g.dst_blocks_i[p] = (int)(((long long)g.n * g.N + lpb - 1) / lpb);
    g.dst_blocks_j[p] = g.n * ((g.N + lpbj - 1) / lpbj);
    int cpb = pow2_floor(std::min(256, std::max(1, budget[p] / lst)));
    cpb = std::max(lpwt, std::min(cpb, pow2_floor(std::max(1, g.m))));
    if (p == 1 && pt) cpb = pipe_time_cols(g.n, g.zeta_pi);
    g.time_cpb[p] = cpb;
    g.time_blocks[p] = (int)(((p == 1 && pt ? g.mp : (long long)g.m) + cpb - 1) / cpb);
    if (p == 1 && (pipe_time_code(g) & 64)) g.time_blocks[p] = g.N * ((g.N + cpb - 1) / cpb);   // rows of points
  }
  matvec_shape(g);
  g.vec_blocks = vec_blocks_for(2 * g.mn);
}

// ---------------------------------------------------------------------------------------------
// Autotuner cache: the winning kernel choices (Geom::tune, dst_q, time_q) per device and problem
// shape, shared by every problem of that shape the process creates afterwards.
// ---------------------------------------------------------------------------------------------
struct TuneKey {
  int dev, N, n, bc, zeta_pi, prec;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, N, n, bc, zeta_pi, prec) < std::tie(o.dev, o.N, o.n, o.bc, o.zeta_pi, o.prec);
  }
};
struct TuneChoice { int tune, dst_q, time_q; };
std::mutex g_tune_mu;
std::map<TuneKey, TuneChoice> g_tune_cache;

TuneKey tune_key(const Geom& g, int prec) {
  int dev = 0;
  cudaGetDevice(&dev);
  return TuneKey{dev, g.N, g.n, g.bc, g.zeta_pi, prec == PCB_MIXED ? 1 : 0};
}

void apply_choice(Geom& g, const TuneChoice& c) {
  g.tune = c.tune; g.dst_q = c.dst_q; g.time_q = c.time_q;
  set_shapes(g);
}

// constant-coefficient problems only: the multigrid route has its own shapes
void apply_cached_tuning(Geom& g, int prec) {
  if (g.mg_route) return;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune_cache.find(tune_key(g, prec));
  if (it != g_tune_cache.end()) apply_choice(g, it->second);
}

}  // namespace

// build a batch descriptor for instances whose Geom/Slots/Scal live in device arrays
static int build_offsets(const std::vector<Geom>& gs, std::vector<int>& host_off, int& tot_out, int which, int p) {
  const int count = (int)gs.size();
  int tot = 0;
  for (int k = 0; k < count; ++k) {
    host_off.push_back(tot);
    const Geom& g = gs[k];
    int nb = 0;
    switch (which) {
      case 0: nb = g.dst_blocks_i[p]; break;
      case 1: nb = g.dst_blocks_j[p]; break;
      case 2: nb = g.time_blocks[p]; break;
      case 3: nb = g.mv_blocks; break;
      default: nb = g.vec_blocks; break;
    }
    tot += nb;
  }
  host_off.push_back(tot);
  tot_out = tot;
  return 0;
}

// Fill B's offset tables for `gs` into the device int buffer `doff` (12 arrays of count+1).
namespace pcb {
int fill_batch(Batch& B, const std::vector<Geom>& gs, int* doff, cudaStream_t st, std::vector<int>& staging) {
  const int count = (int)gs.size();
  staging.clear();
  int tots[8];
  // order: dst_i[0], dst_i[1], dst_j[0], dst_j[1], time[0], time[1], mv, vec
  const int which[8] = {0, 0, 1, 1, 2, 2, 3, 4};
  const int prec[8] = {0, 1, 0, 1, 0, 1, 0, 0};
  for (int a = 0; a < 8; ++a) build_offsets(gs, staging, tots[a], which[a], prec[a]);
  CK(cudaMemcpyAsync(doff, staging.data(), staging.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  const int stride = count + 1;
  for (int p = 0; p < 2; ++p) {
    B.off_dst_i[p] = doff + (0 + p) * stride; B.tot_dst_i[p] = tots[0 + p];
    B.off_dst_j[p] = doff + (2 + p) * stride; B.tot_dst_j[p] = tots[2 + p];
    B.off_time[p] = doff + (4 + p) * stride;  B.tot_time[p] = tots[4 + p];
    B.dst_smem[p] = 0; B.time_smem[p] = 0;
    for (const Geom& g : gs) {
      B.dst_smem[p] = std::max(B.dst_smem[p], dst_smem_bytes(g, p));
      B.time_smem[p] = std::max(B.time_smem[p], time_smem_bytes(g, p));
    }
  }
  B.off_mv = doff + 6 * stride; B.tot_mv = tots[6];
  B.off_vec = doff + 7 * stride; B.tot_vec = tots[7];
  B.count = count;
  B.stream = st;
  B.fem_m = count == 1 && gs[0].fem ? gs[0].m : 0;
  {
    int want = -1;     // the n = 512 zeta = pi time pass variant, when all its instances agree
    for (const Geom& g : gs) {
      if (!g.time_blocks[1] || pipe_time_p(g) != 16 || !g.zeta_pi) continue;
      const int v = (g.tune & TUNE_TIME512_3BLK) ? 1 : (g.tune & TUNE_TIME512_4BLK) ? 2 : 0;
      want = want < 0 ? v : (want == v ? v : 0);
    }
    B.t512v = want > 0 ? want : 0;
  }
  B.dst_q = gs[0].dst_q;
  B.time_q = gs[0].time_q;
  for (const Geom& g : gs) {   // mixed sizes: shared launches dispatch per instance
    if (g.dst_q != B.dst_q) B.dst_q = 0;
    if (g.time_q != B.time_q) B.time_q = 0;
  }
  // FP32 kernel families (pipelined P or 0) of the instances with work (empty server slots have none)
  const size_t fam_at = staging.size();
  B.fam_dst_set = B.fam_time_set = 0;
  for (const Geom& g : gs) staging.push_back(pipe_dst_code(g));
  for (const Geom& g : gs) staging.push_back(pipe_time_code(g));
  for (const Geom& g : gs) {
    if (g.dst_blocks_i[1] > 0) B.fam_dst_set |= 1 << fam_index(pipe_dst_code(g));
    if (g.time_blocks[1] > 0) B.fam_time_set |= 1 << fam_index(pipe_time_code(g));
  }
  auto uniform = [](int set) {
    return __builtin_popcount(set) == 1 ? fam_code(__builtin_ctz(set)) : (set ? -1 : 0);
  };
  B.pipe_pd = uniform(B.fam_dst_set);
  B.pipe_pt = uniform(B.fam_time_set);
  B.fam_dst = doff + fam_at;
  B.fam_time = doff + fam_at + count;
  B.filt = nullptr;
  B.filt_want = 0;
  CK(cudaMemcpyAsync(doff + fam_at, staging.data() + fam_at, 2 * count * sizeof(int), cudaMemcpyHostToDevice, st));
  return PCB_OK;
}
}  // namespace pcb

extern "C" {

const char* pcb_status_str(int s) {
  switch (s) {
    case PCB_OK: return "ok";
    case PCB_NOT_CONVERGED: return "not converged (maximum iterations reached)";
    case PCB_ERR_INVALID_ARG: return "invalid argument";
    case PCB_ERR_UNSUPPORTED: return "unsupported configuration";
    case PCB_ERR_SINGULAR: return "singular preconditioner factor";
    case PCB_ERR_OUT_OF_MEMORY: return "out of device memory";
    case PCB_ERR_CUDA: return "CUDA runtime error";
    case PCB_ERR_NONFINITE: return "non-finite value";
    case PCB_ERR_BREAKDOWN: return "Krylov breakdown";
    case PCB_ERR_TIMEOUT: return "device wait timed out";
    case PCB_ERR_TOO_LARGE: return "request exceeds size limit";
    default: return "unknown status";
  }
}

long long pcb_unknowns(const pcb_problem* p) { return p ? 2 * p->g.mn : 0; }
long long pcb_workspace_bytes(const pcb_problem* p) { return p ? p->bytes : 0; }

void pcb_destroy(pcb_problem* p) {
  if (!p) return;
  cudaStreamSynchronize(p->stream);
  cudaFree(p->tables);
  cudaFree(p->scratch);
  if (p->mgws) mg_release(p->mgws);
  cudaFree(p->mgws);
  cudaFree(p->vec_minres);
  cudaFree(p->vec_mixed);
  cudaFree(p->vec_gmres);
  cudaFree(p->dG);
  cudaFree(p->dS);
  cudaFree(p->dSc);
  cudaFree(p->doff);
  cudaFree(p->partial);
  cudaFreeHost(p->hSc);
  cudaFreeHost(p->hSpin);
  cudaFree(p->host_io);
  if (p->git) cudaGraphExecDestroy(p->git);
  for (cudaGraphExec_t e : p->garn) if (e) cudaGraphExecDestroy(e);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  cudaFree(p->dtol);
  for (cudaEvent_t e : p->ev_prec) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_mv) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_mvi) cudaEventDestroy(e);
  delete p;
}

}  // extern "C"

namespace pcb {

// Validation shared by every entry point that takes a descriptor.
int validate_desc(const pcb_desc* d) {
  if (!d) return PCB_ERR_INVALID_ARG;
  if (d->N < 1 || d->n < 2 || !(d->theta >= 0.5 && d->theta <= 1.0) || !(d->gamma > 0.0) || !(d->T > 0.0) ||
      (d->precision != PCB_FP64 && d->precision != PCB_MIXED) || !std::isfinite(d->zeta) ||
      !std::isfinite(d->gamma) || !std::isfinite(d->T))
    return PCB_ERR_INVALID_ARG;
  if (d->bc != PCB_BC_DIRICHLET && d->bc != PCB_BC_NEUMANN) return PCB_ERR_INVALID_ARG;
  if (!std::isfinite(d->a_const)) return PCB_ERR_INVALID_ARG;
  const bool neu = d->bc == PCB_BC_NEUMANN;
  // supported: any zeta (multigrid route: zeta = pi), n a power of two <= 1024; Dirichlet
  // N+1 = 2^a 3^b with N <= 511, Neumann N-1 = 2^a 3^b with 3 <= N <= 513 and constant a
  if (d->a_edges && std::fabs(d->zeta - M_PI) > 1e-12) return PCB_ERR_UNSUPPORTED;
  if (!pow2(d->n) || d->n > 1024) return PCB_ERR_UNSUPPORTED;
  if (neu ? (d->N < 3 || d->N > 513 || d->a_edges) : d->N > 511) return PCB_ERR_UNSUPPORTED;
  const int M = neu ? 2 * (d->N - 1) : 2 * (d->N + 1);
  FftPlan pd, pt;
  if (!make_plan(M, pd) || !make_plan(d->n, pt)) return PCB_ERR_UNSUPPORTED;
  if (!q_supported(dst_Q(M)) || !q_supported(time_Q(d->n))) return PCB_ERR_UNSUPPORTED;
  if (d->a_edges && !pow2(d->N + 1)) return PCB_ERR_UNSUPPORTED;
  if (d->a_edges && !mg_available()) return PCB_ERR_UNSUPPORTED;
  if (d->a_edges && d->n > 512) return PCB_ERR_UNSUPPORTED;
  if (d->fem != 0 && d->fem != 1) return PCB_ERR_INVALID_ARG;
  if (d->fem && (neu || d->a_edges)) return PCB_ERR_UNSUPPORTED;
  if (d->multigrid != 0 && d->multigrid != 1) return PCB_ERR_INVALID_ARG;
  if (d->multigrid && !d->a_edges) {
    // the multigrid route with a constant coefficient: Dirichlet N = 2^k - 1, Neumann N = 2^k + 1
    if (d->fem || std::fabs(d->zeta - M_PI) > 1e-12 || d->n > 512 || !mg_available()) return PCB_ERR_UNSUPPORTED;
    if (neu ? (d->N < 5 || !pow2(d->N - 1)) : !pow2(d->N + 1)) return PCB_ERR_UNSUPPORTED;
  }
  if (d->a_edges) {
    const long long ne = 2LL * d->N * (d->N + 1);
    for (long long k = 0; k < ne; ++k)
      if (!(d->a_edges[k] > 0.0) || !std::isfinite(d->a_edges[k])) return PCB_ERR_INVALID_ARG;
  }
  return PCB_OK;
}

// Scalar fields, FFT plans and launch shapes of a validated descriptor (no device work).
void init_geom(const pcb_desc* d, Geom& g) {
  std::memset(&g, 0, sizeof(g));
  g.bc = d->bc == PCB_BC_NEUMANN ? PCB_BC_NEUMANN : PCB_BC_DIRICHLET;
  const bool neu = g.bc == PCB_BC_NEUMANN;
  g.N = d->N; g.n = d->n; g.m = d->N * d->N; g.L = neu ? d->N - 1 : d->N + 1; g.M = 2 * g.L;
  g.mn = (long long)g.m * g.n;
  g.theta = d->theta; g.tau = d->T / d->n; g.gamma = d->gamma; g.alpha = g.tau / std::sqrt(d->gamma);
  g.h = 1.0 / g.L; g.sqrt_gamma = std::sqrt(d->gamma);
  const double a0 = d->a_const > 0.0 ? d->a_const : 1.0;
  g.c = a0 * g.tau / (g.h * g.h);
  g.var_a = d->a_edges ? 1 : 0;
  g.mg_route = d->a_edges || d->multigrid ? 1 : 0;
  g.fem = d->fem ? 1 : 0;
  g.zeta = d->zeta;
  g.zeta_pi = std::fabs(d->zeta - M_PI) <= 1e-12 ? 1 : 0;
  make_plan(g.M, g.pdst);
  make_plan(g.n, g.ptime);
  g.dst_q = dst_Q(g.M);
  g.time_q = time_Q(g.n);
  set_shapes(g);
}

// Byte offsets of the spectral / twiddle / coefficient tables (Sec. 3.5) inside one buffer.
size_t table_layout(const Geom& g, TableLayout& t) {
  const int N = g.N, n = g.n, M = g.M;
  const size_t ne = g.var_a ? (size_t)N * (N + 1) : 0;
  size_t off_b = 0;
  auto take = [&](size_t bytes) { size_t o = off_b; off_b += (bytes + 255) & ~(size_t)255; return o; };
  t.kap = take((size_t)N * 8); t.mud = take((size_t)n * 16); t.muf = take((size_t)n * 8);
  t.twdd = take((size_t)M * 16); t.twdf = take((size_t)M * 8); t.twtd = take((size_t)n * 16);
  t.twtf = take((size_t)n * 8); t.pred = take((size_t)n * 16); t.pref = take((size_t)n * 8);
  t.ax = take(ne * 8); t.ay = take(ne * 8); t.dg = take(g.var_a ? (size_t)g.m * 8 : 0);
  t.ms = take(g.fem ? (size_t)N * 8 : 0);
  t.bytes = off_b;
  return off_b;
}

// Fill the tables (FP64 on the host with the C math library, rounded for the FP32 copies).
void fill_tables(const pcb_desc* d, const Geom& g, const TableLayout& t, unsigned char* host) {
  const int N = g.N, n = g.n, M = g.M;
  std::memset(host, 0, t.bytes);
  double* kap = (double*)(host + t.kap);
  const double a0 = d->a_const > 0.0 && !d->a_edges ? d->a_const : 1.0;
  for (int q = 0; q < N; ++q) {
    // Dirichlet mode q+1 of the DST-I, Neumann mode q of the DCT-I: a (4/h^2) sin^2(k pi / (2L))
    const int k = g.bc == PCB_BC_NEUMANN ? q : q + 1;
    const double s = std::sin(k * M_PI / (2.0 * g.L));
    kap[q] = a0 * 4.0 / (g.h * g.h) * s * s;
    if (g.fem) {
      // linear elements: K1 = (1/h) tridiag(-1, 2, -1) and M1 = (h/6) tridiag(1, 4, 1) share the sine
      // modes; kappa1 = (4/h) sin^2(k pi h/2), mu = (h/6)(4 + 2 cos(k pi h)); M1^{-1/2} K1 M1^{-1/2}
      // has the eigenvalues kappa1/mu
      const double mu = g.h / 6.0 * (4.0 + 2.0 * std::cos(k * M_PI * g.h));
      ((double*)(host + t.ms))[q] = mu;
      kap[q] = a0 * (4.0 / g.h) * s * s / mu;
    }
  }
  // lambda(S_n) at F-slot r: psi_r = -(zeta + 2 pi r)/n (zeta = pi: -pi (2r+1)/n), f1/f2 with
  // f1 = 1 - e^{i psi}, f2 = theta + (1-theta) e^{i psi}
  double2* mud = (double2*)(host + t.mud);
  float2* muf = (float2*)(host + t.muf);
  for (int r = 0; r < n; ++r) {
    const double psi = g.zeta_pi ? -M_PI * (2.0 * r + 1.0) / n : -(g.zeta + 2.0 * M_PI * r) / n;
    const double c = std::cos(psi), s = std::sin(psi);
    const double f1r = 1.0 - c, f1i = -s;
    double f2r = g.theta + (1.0 - g.theta) * c, f2i = (1.0 - g.theta) * s;
    if (std::hypot(f2r, f2i) < 1e-14) { f2r = 1.0; f2i = 0.0; }   // Remark 1 remedy (theta = 1/2, psi = pi)
    const double den = f2r * f2r + f2i * f2i;
    mud[r].x = (f1r * f2r + f1i * f2i) / den;
    mud[r].y = (f1i * f2r - f1r * f2i) / den;
    muf[r].x = (float)mud[r].x; muf[r].y = (float)mud[r].y;
  }
  auto fill_tw = [&](double2* td, float2* tf, int len) {
    for (int k = 0; k < len; ++k) {
      const double a = -2.0 * M_PI * (double)k / (double)len;
      td[k].x = std::cos(a); td[k].y = std::sin(a);
      tf[k].x = (float)td[k].x; tf[k].y = (float)td[k].y;
    }
  };
  fill_tw((double2*)(host + t.twdd), (float2*)(host + t.twdf), M);
  fill_tw((double2*)(host + t.twtd), (float2*)(host + t.twtf), n);
  double2* pred = (double2*)(host + t.pred);
  float2* pref = (float2*)(host + t.pref);
  for (int k = 0; k < n; ++k) {
    const double a = (g.zeta_pi ? -M_PI : -g.zeta) * (double)k / n;   // exp(-i zeta t / n)
    pred[k].x = std::cos(a); pred[k].y = std::sin(a);
    pref[k].x = (float)pred[k].x; pref[k].y = (float)pred[k].y;
  }
  if (g.var_a) {
    const size_t ne = (size_t)N * (N + 1);
    double* ax = (double*)(host + t.ax);
    double* ay = (double*)(host + t.ay);
    double* dg = (double*)(host + t.dg);
    const double* axs = d->a_edges;
    const double* ays = d->a_edges + ne;
    for (size_t k = 0; k < ne; ++k) { ax[k] = g.c * axs[k]; ay[k] = g.c * ays[k]; }
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i)
        dg[j * N + i] = ax[j * (N + 1) + i] + ax[j * (N + 1) + i + 1] + ay[j * N + i] + ay[(j + 1) * N + i];
  }
}

// Point the Geom's table pointers into a device copy of the tables.
void bind_tables(Geom& g, const TableLayout& t, unsigned char* tb) {
  g.kap = (const double*)(tb + t.kap);
  g.mu_d = (const double2*)(tb + t.mud); g.mu_f = (const float2*)(tb + t.muf);
  g.twd_d = (const double2*)(tb + t.twdd); g.twd_f = (const float2*)(tb + t.twdf);
  g.twt_d = (const double2*)(tb + t.twtd); g.twt_f = (const float2*)(tb + t.twtf);
  g.pre_d = (const double2*)(tb + t.pred); g.pre_f = (const float2*)(tb + t.pref);
  if (g.var_a) {
    g.axs = (const double*)(tb + t.ax); g.ays = (const double*)(tb + t.ay); g.dgs = (const double*)(tb + t.dg);
  }
  g.mass = g.fem ? (const double*)(tb + t.ms) : nullptr;
}

}  // namespace pcb

extern "C" {

int pcb_create(const pcb_desc* d_in, pcb_problem** out) {
  if (!d_in || !out) return PCB_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = validate_desc(d_in);
  if (rc != PCB_OK) return rc;
  // Dirichlet with multigrid requested for a constant coefficient: the variable-coefficient route
  // with every edge value equal to a (the same operator)
  pcb_desc dd = *d_in;
  std::vector<double> const_edges;
  if (dd.multigrid && !dd.a_edges && dd.bc != PCB_BC_NEUMANN) {
    const_edges.assign((size_t)2 * dd.N * (dd.N + 1), dd.a_const > 0.0 ? dd.a_const : 1.0);
    dd.a_edges = const_edges.data();
    dd.a_const = 0.0;      // the edge values carry a (the stencil scale is then tau/h^2)
  }
  const pcb_desc* d = &dd;
  pcb_problem* p = new (std::nothrow) pcb_problem();
  if (!p) return PCB_ERR_OUT_OF_MEMORY;
  p->desc = *d;
  p->desc.a_edges = nullptr;
  if (p->desc.mg_cycles <= 0) p->desc.mg_cycles = 2;
  p->stream = (cudaStream_t)d->stream;
  cudaGetDevice(&p->device);
  Geom& g = p->g;
  init_geom(d, g);
  apply_cached_tuning(g, d->precision);
  if (upload_constants() != cudaSuccess) { delete p; return PCB_ERR_CUDA; }
  auto fail = [&](int code) { pcb_destroy(p); return code; };
  TableLayout lay;
  const size_t off_b = table_layout(g, lay);
  std::vector<unsigned char> host(off_b, 0);
  fill_tables(d, g, lay, host.data());
  if (cudaMalloc(&p->tables, off_b) != cudaSuccess) return fail(PCB_ERR_OUT_OF_MEMORY);
  p->bytes += off_b;
  if (cudaMemcpy(p->tables, host.data(), off_b, cudaMemcpyHostToDevice) != cudaSuccess) return fail(PCB_ERR_CUDA);
  bind_tables(g, lay, (unsigned char*)p->tables);
  // ---- preconditioner scratch: 2mn values, FP64-sized so both precisions fit ----
  // (the pipelined FP32 passes keep two buffers of padded rows in it: 16 n N lr bytes)
  // (sized for the padded layout of the pipelined passes even when a tuned choice does not use it,
  // so that pcb_autotune may try every kernel family on this problem)
  const size_t sbytes = std::max<size_t>((size_t)2 * g.mn * sizeof(double), (size_t)16 * g.n * g.N * (size_t)(g.L + 16));
  if (cudaMalloc(&p->scratch, sbytes) != cudaSuccess) return fail(PCB_ERR_OUT_OF_MEMORY);
  p->bytes += sbytes;
  g.scratch = p->scratch;
  if (g.mg_route) {
    const size_t mb = mg_workspace_bytes(g);
    if (cudaMalloc(&p->mgws, mb) != cudaSuccess) return fail(PCB_ERR_OUT_OF_MEMORY);
    p->bytes += mb;
    if (mg_setup(g, p->mgws, d->a_edges, d->a_const > 0.0 ? d->a_const : 1.0) != cudaSuccess) return fail(PCB_ERR_CUDA);
  }
  // ---- single-instance batch ----
  if (cudaMalloc(&p->dG, sizeof(Geom)) != cudaSuccess || cudaMalloc(&p->dS, sizeof(Slots)) != cudaSuccess ||
      cudaMalloc(&p->dSc, sizeof(Scal)) != cudaSuccess || cudaMalloc(&p->doff, 10 * 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&p->partial, (size_t)g.vec_blocks * (PCB_MAX_RESTART + 2) * sizeof(double) +
                                  (size_t)std::max(g.mv_blocks, 1) * sizeof(double)) != cudaSuccess)
    return fail(PCB_ERR_OUT_OF_MEMORY);
  if (cudaMallocHost(&p->hSc, sizeof(Scal)) != cudaSuccess || cudaMallocHost(&p->hSpin, sizeof(Slots)) != cudaSuccess)
    return fail(PCB_ERR_OUT_OF_MEMORY);
  std::memset(&p->hS, 0, sizeof(Slots));
  if (cudaMemcpy(p->dG, &g, sizeof(Geom), cudaMemcpyHostToDevice) != cudaSuccess) return fail(PCB_ERR_CUDA);
  if (cudaMemset(p->dSc, 0, sizeof(Scal)) != cudaSuccess) return fail(PCB_ERR_CUDA);
  std::vector<Geom> gs(1, g);
  std::vector<int> staging;
  std::memset(&p->B, 0, sizeof(Batch));
  if ((rc = fill_batch(p->B, gs, p->doff, p->stream, staging)) != PCB_OK) return fail(rc);
  if (cudaStreamSynchronize(p->stream) != cudaSuccess) return fail(PCB_ERR_CUDA);   // staging is read
  p->B.G = p->dG; p->B.S = p->dS; p->B.Sc = p->dSc; p->B.active = nullptr; p->B.partial = p->partial;
  p->B.stream = p->stream;
  *out = p;
  return PCB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// slot upload (single instance): pinned staging + async copy on the problem stream
// ---------------------------------------------------------------------------------------------
static int upload_slots(pcb_problem* p) {
  CK(cudaStreamSynchronize(p->stream));   // the pinned staging buffer may still be in flight
  *p->hSpin = p->hS;
  CK(cudaMemcpyAsync(p->dS, p->hSpin, sizeof(Slots), cudaMemcpyHostToDevice, p->stream));
  return PCB_OK;
}

static int ensure_minres(pcb_problem* p) {
  if (p->vec_minres) return PCB_OK;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  if (cudaMalloc(&p->vec_minres, 7 * vb) != cudaSuccess) { cudaGetLastError(); p->vec_minres = nullptr; return PCB_ERR_OUT_OF_MEMORY; }
  p->bytes += 7 * vb;
  return PCB_OK;
}
static int ensure_mixed(pcb_problem* p) {
  if (p->vec_mixed) return PCB_OK;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  if (cudaMalloc(&p->vec_mixed, 2 * vb) != cudaSuccess) { cudaGetLastError(); p->vec_mixed = nullptr; return PCB_ERR_OUT_OF_MEMORY; }
  p->bytes += 2 * vb;
  return PCB_OK;
}
static int ensure_gmres(pcb_problem* p, int restart) {
  if (p->vec_gmres && p->gmres_restart >= restart) return PCB_OK;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  if (p->vec_gmres) { cudaStreamSynchronize(p->stream); cudaFree(p->vec_gmres); p->bytes -= (long long)(2 * p->gmres_restart + 2) * vb; p->vec_gmres = nullptr; }
  if (cudaMalloc(&p->vec_gmres, (size_t)(2 * restart + 2) * vb) != cudaSuccess) { cudaGetLastError(); p->vec_gmres = nullptr; return PCB_ERR_OUT_OF_MEMORY; }
  p->gmres_restart = restart;
  p->bytes += (long long)(2 * restart + 2) * vb;
  return PCB_OK;
}

// ---------------------------------------------------------------------------------------------
// the solvers (operate on a Batch; the single-instance API is a batch of one)
// ---------------------------------------------------------------------------------------------
struct SolveCfg {
  int op, prec, kind, method, maxit, restart, fixed;
  double tol;
  double inner_floor;   // mixed precision: smallest inner tolerance
  bool check_true;      // FP64 route: keep iterating if the true residual check fails
  bool graphs;          // replay MINRES iterations from a captured CUDA graph
};

static int apply_precond(const pcb_problem* p, const Batch& B, int kind, int prec, int in_slot, int out_slot) {
  cudaError_t e;
  if (kind == PCB_PREC_NONE) e = launch_axpby(B, AX_COPY, in_slot, out_slot, -1);
  else if (p->g.mg_route) e = launch_precond_mg(B, p->g, kind, prec, p->desc.mg_cycles, in_slot, out_slot);
  else e = launch_precond_fast(B, kind, prec, in_slot, out_slot);
  return e == cudaSuccess ? PCB_OK : cuda_status(e);
}

namespace pcb { int precond_launch_count(bool var_a, int kind); }

// event pair from a pool (grown on demand); returns false when profiling is off
static bool ev_pair(std::vector<cudaEvent_t>& pool, int& used, cudaEvent_t& a, cudaEvent_t& b) {
  if ((int)pool.size() < 2 * (used + 1)) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return false;
      pool.push_back(e);
    }
  }
  a = pool[2 * used]; b = pool[2 * used + 1];
  ++used;
  return true;
}

static int P_precond(pcb_problem* p, const Batch& B, int kind, int prec, int in_slot, int out_slot) {
  const bool va = p->g.mg_route != 0;
  cudaEvent_t a = nullptr, b = nullptr;
  const bool ev = p->prof && ev_pair(p->ev_prec, p->ev_prec_used, a, b);
  if (ev) cudaEventRecord(a, B.stream);
  const long long mg0 = mg_launch_total();
  const int rc = apply_precond(p, B, kind, prec, in_slot, out_slot);
  if (ev) cudaEventRecord(b, B.stream);
  p->launches += va ? (mg_launch_total() - mg0) : precond_launch_count(va, kind);
  p->prec_applies += 1;
  return rc;
}

static cudaError_t P_matvec(pcb_problem* p, const Batch& B, int op, int x_slot, int out_slot, int aux_slot, int epi) {
  cudaEvent_t a = nullptr, b = nullptr;
  const bool inner = (epi & EPI_FAST) != 0;
  const bool ev = p->prof && (inner ? ev_pair(p->ev_mvi, p->ev_mvi_used, a, b) : ev_pair(p->ev_mv, p->ev_mv_used, a, b));
  if (ev) cudaEventRecord(a, B.stream);
  const cudaError_t e = launch_matvec(B, op, x_slot, out_slot, aux_slot, epi);
  if (ev) cudaEventRecord(b, B.stream);
  p->launches += 1;
  p->matvecs += 1;
  p->matvecs_inner += inner ? 1 : 0;
  return e;
}

static double ev_sum(const std::vector<cudaEvent_t>& pool, int used) {
  double s = 0.0;
  for (int k = 0; k < used; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pool[2 * k], pool[2 * k + 1]) == cudaSuccess) s += ms;
  }
  return s;
}

// Poll per-instance scalars (synchronises the stream).
static int read_scal(const Batch& B, Scal* host, int count) {
  CK(cudaMemcpyAsync(host, B.Sc, sizeof(Scal) * count, cudaMemcpyDeviceToHost, B.stream));
  CK(cudaStreamSynchronize(B.stream));
  return PCB_OK;
}

// Single-instance MINRES on slot rhs -> slot x (both set by the caller).  Returns iterations via sc.
#define LC(p) (++(p)->launches, 0) ? cudaSuccess :

// One MINRES iteration's launches: product with the Lanczos epilogue, scalar steps, residual
// update, preconditioner, inner product, direction/solution update, slot rotation.  Every kernel
// takes its scalars and vector pointers from device memory (Scal, Slots, the tolerance in
// B.tols), so one launch sequence serves every iteration and can be replayed from a graph.
static int minres_iter_launches(pcb_problem* p, const Batch& B, const SolveCfg& c, int s_x) {
  int rc;
  CK(P_matvec(p, B, PCB_OP_A, SL_Y, SL_Q, SL_R1, EPI_MINRES | (c.prec == PCB_MIXED ? EPI_FAST : 0)));
  CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_MINRES_ALFA, c.tol, 0, 0));
  CK(LC(p) launch_axpby(B, AX_MINRES_R, SL_Q, SL_R2, SL_R1));
  if ((rc = P_precond(p, B, c.kind, c.prec, SL_R1, SL_YO))) return rc;
  CK(LC(p) launch_dot(B, SL_R1, SL_YO));
  CK(LC(p) launch_reduce(B, B.off_vec, 1, 0, SS_MINRES_GIVENS, c.tol, 0, 0));
  CK(LC(p) launch_minres_wx(B, SL_Y, SL_W, SL_W2, s_x));
  CK(LC(p) launch_swap(B, SL_R1, SL_R2, SL_Y, SL_YO, SL_W, SL_W2));
  return PCB_OK;
}

// Capture minres_iter_launches into p->git (on a private stream: the caller's may be the legacy
// default stream, which cannot be captured).  Returns false when capture is not possible; the
// caller then launches directly.  Counters are restored: the captured launches did not run.
// Capture the launches `issue(Bc)` makes on a private stream into an executable graph (null when
// capture is not possible).  *launches gets the kernel count; the counters are restored, since
// the captured launches did not run.
template <typename F>
static cudaGraphExec_t capture_launches(pcb_problem* p, const Batch& B, F&& issue, long long* launches) {
  if (!p->cap_stream && cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError(); p->cap_stream = nullptr; return nullptr;
  }
  Batch Bc = B;
  Bc.stream = p->cap_stream;
  const long long l0 = p->launches;
  const int a0 = p->prec_applies, m0 = p->matvecs, mi0 = p->matvecs_inner;
  if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError(); return nullptr;
  }
  const int rc = issue(Bc);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
  *launches = p->launches - l0;
  p->launches = l0; p->prec_applies = a0; p->matvecs = m0; p->matvecs_inner = mi0;
  if (rc != PCB_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return exec;
}

static bool capture_minres_iter(pcb_problem* p, const Batch& B, const SolveCfg& c, int s_x) {
  if (p->git) { cudaGraphExecDestroy(p->git); p->git = nullptr; }
  p->git = capture_launches(p, B, [&](const Batch& Bc) { return minres_iter_launches(p, Bc, c, s_x); },
                            &p->git_launches);
  if (!p->git) return false;
  p->git_kind = c.kind; p->git_prec = c.prec; p->git_sx = s_x;
  return true;
}

static int minres_single(pcb_problem* p, const SolveCfg& c, int s_b, int s_x, Scal* hs, double* relres_out,
                         int* it_out, bool* conv_out) {
  const Batch& B = p->B;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  // x = 0, w = w2 = 0, r1 = r2 = b
  CK(cudaMemsetAsync(p->hS.v[s_x], 0, vb, p->stream));
  CK(cudaMemsetAsync(p->hS.v[SL_W], 0, vb, p->stream));
  CK(cudaMemsetAsync(p->hS.v[SL_W2], 0, vb, p->stream));
  CK(LC(p) launch_axpby(B, AX_COPY, s_b, SL_R1, -1));
  CK(LC(p) launch_axpby(B, AX_COPY, s_b, SL_R2, -1));
  CK(LC(p) launch_dot(B, s_b, s_b));
  CK(LC(p) launch_reduce(B, B.off_vec, 1, 0, SS_BNORM, c.tol, 0, 0));
  int rc = P_precond(p, B, c.kind, c.prec, SL_R2, SL_Y);
  if (rc) return rc;
  CK(LC(p) launch_dot(B, SL_R2, SL_Y));
  CK(LC(p) launch_reduce(B, B.off_vec, 1, 0, SS_MINRES_INIT, c.tol, 0, 0));
  if ((rc = read_scal(B, hs, 1))) return rc;
  *it_out = 0; *conv_out = false; *relres_out = 1.0;
  if (hs->flags & 4) return PCB_ERR_NONFINITE;
  if (hs->flags & 2) return PCB_ERR_BREAKDOWN;
  if (hs->bnorm == 0.0 || !hs->active) { *conv_out = true; *relres_out = 0.0; return PCB_OK; }
  const int limit = c.fixed > 0 ? c.fixed : c.maxit;
  bool checking = false;
  // the iterations read the tolerance from the device, so a captured graph serves every sweep
  if (!p->dtol && cudaMalloc(&p->dtol, sizeof(double)) != cudaSuccess) { cudaGetLastError(); p->dtol = nullptr; }
  Batch Bt = B;
  bool graph = c.graphs && !p->prof && p->dtol;
  if (p->dtol) {
    CK(cudaMemcpyAsync(p->dtol, &c.tol, sizeof(double), cudaMemcpyHostToDevice, p->stream));
    Bt.tols = p->dtol;
  }
  for (int it = 0; it < limit; ++it) {
    // the first iteration runs directly (one-time kernel attribute setup happens there)
    if (graph && it >= 1 && !(p->git && p->git_kind == c.kind && p->git_prec == c.prec && p->git_sx == s_x))
      graph = capture_minres_iter(p, Bt, c, s_x);
    if (graph && it >= 1) {
      CK(cudaGraphLaunch(p->git, p->stream));
      p->launches += p->git_launches;
      p->prec_applies += 1;
      p->matvecs += 1;
      p->matvecs_inner += c.prec == PCB_MIXED ? 1 : 0;
    } else if ((rc = minres_iter_launches(p, Bt, c, s_x))) {
      return rc;
    }
    std::swap(p->hS.v[SL_R1], p->hS.v[SL_R2]);
    std::swap(p->hS.v[SL_Y], p->hS.v[SL_YO]);
    std::swap(p->hS.v[SL_W], p->hS.v[SL_W2]);
    if ((rc = read_scal(B, hs, 1))) return rc;
    *it_out = it + 1;
    if (hs->flags & 4) return PCB_ERR_NONFINITE;
    if (hs->flags & 2) return PCB_ERR_BREAKDOWN;
    if (c.fixed > 0) continue;
    if ((hs->flags & 1) || checking) {
      // an inner solve of a refinement sweep ends at its first estimate below the tolerance; the
      // sweep then measures the true residual of the outer system itself
      if (!c.check_true) { *relres_out = hs->est; return PCB_OK; }
      CK(P_matvec(p, B, PCB_OP_A, s_x, SL_Q, s_b, EPI_RESID));
      CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
      if ((rc = read_scal(B, hs, 1))) return rc;
      const double rel = std::sqrt(hs->dot1) / hs->bnorm;
      *relres_out = rel;
      if (rel <= c.tol) { *conv_out = true; return PCB_OK; }
      checking = true;
    }
  }
  if (!c.check_true) { *relres_out = hs->est; return PCB_OK; }
  CK(P_matvec(p, B, PCB_OP_A, s_x, SL_Q, s_b, EPI_RESID));
  CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
  if ((rc = read_scal(B, hs, 1))) return rc;
  *relres_out = std::sqrt(hs->dot1) / hs->bnorm;
  *conv_out = *relres_out <= c.tol;
  return PCB_OK;
}

// Arnoldi step j of FGMRES: z_j = P^-1 v_j, w = op z_j, two classical Gram-Schmidt passes,
// ||w||, the Hessenberg column and its rotations (scalar step), v_{j+1} = w/||w||.  All operands
// come from device memory (slots, scalars, the tolerance in B.tols), so a graph per j serves every
// restart cycle and solve with the same setting.
static int arnoldi_launches(pcb_problem* p, const Batch& B, const SolveCfg& c, int j) {
  int rc;
  const int op = PCB_OP_AHAT;
  CK(LC(p) launch_setslot(B, SL_VJ, SL_VBASE, j));
  CK(LC(p) launch_setslot(B, SL_ZJ, SL_ZBASE, j));
  CK(LC(p) launch_setslot(B, SL_VJ1, SL_VBASE, j + 1));
  if ((rc = P_precond(p, B, c.kind, c.prec, SL_VJ, SL_ZJ))) return rc;
  CK(P_matvec(p, B, op, SL_ZJ, SL_VJ1, -1, EPI_PLAIN));
  for (int pass = 0; pass < 2; ++pass) {
    CK(LC(p) launch_multidot(B, SL_VBASE, j, SL_VJ1));
    CK(LC(p) launch_reduce_multi(B, j, pass));
    CK(LC(p) launch_multiaxpy(B, SL_VBASE, j, SL_VJ1, pass));
  }
  CK(LC(p) launch_dot(B, SL_VJ1, SL_VJ1));
  CK(LC(p) launch_reduce(B, B.off_vec, 1, 0, SS_GMRES_ARNOLDI, c.tol, j, c.restart));
  CK(LC(p) launch_axpby(B, AX_SCALE_INV_HNORM, SL_VJ1, SL_VJ1, -1));
  return PCB_OK;
}

static int fgmres_single(pcb_problem* p, const SolveCfg& c, int s_b, int s_x, Scal* hs, double* relres_out,
                         int* it_out, bool* conv_out) {
  const Batch& B = p->B;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  const int op = PCB_OP_AHAT;
  CK(cudaMemsetAsync(p->hS.v[s_x], 0, vb, p->stream));
  CK(cudaMemsetAsync(p->dSc, 0, sizeof(Scal), p->stream));
  CK(LC(p) launch_dot(B, s_b, s_b));
  CK(LC(p) launch_reduce(B, B.off_vec, 1, 0, SS_BNORM, c.tol, 0, 0));
  int rc;
  if ((rc = read_scal(B, hs, 1))) return rc;
  *it_out = 0; *conv_out = false; *relres_out = 1.0;
  if (!std::isfinite(hs->bnorm)) return PCB_ERR_NONFINITE;
  if (hs->bnorm == 0.0) { *conv_out = true; *relres_out = 0.0; return PCB_OK; }
  const int limit = c.fixed > 0 ? c.fixed : c.maxit;
  int total = 0;
  // Arnoldi steps replay per-j graphs (the first j = 0 step of a solve runs directly)
  if (!p->dtol && cudaMalloc(&p->dtol, sizeof(double)) != cudaSuccess) { cudaGetLastError(); p->dtol = nullptr; }
  Batch Bt = B;
  const bool graph = c.graphs && !p->prof && p->dtol;
  if (p->dtol) {
    CK(cudaMemcpyAsync(p->dtol, &c.tol, sizeof(double), cudaMemcpyHostToDevice, p->stream));
    Bt.tols = p->dtol;
  }
  if (graph && !(p->garn_kind == c.kind && p->garn_prec == c.prec && p->garn_restart == c.restart)) {
    for (cudaGraphExec_t& e : p->garn) if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    p->garn_kind = c.kind; p->garn_prec = c.prec; p->garn_restart = c.restart;
  }
  bool direct_first = true;
  while (total < limit) {
    CK(P_matvec(p, B, op, s_x, SL_R, s_b, EPI_RESID));
    CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_GMRES_START, c.tol, 0, 0));
    if ((rc = read_scal(B, hs, 1))) return rc;
    if (hs->flags & 4) return PCB_ERR_NONFINITE;
    *relres_out = hs->est;
    if (c.fixed <= 0 && hs->est <= c.tol) { *conv_out = true; return PCB_OK; }
    CK(LC(p) launch_setslot(B, SL_VJ, SL_VBASE, 0));
    CK(LC(p) launch_axpby(B, AX_SCALE_INV_BETA, SL_R, SL_VJ, -1));
    const int mres = std::min(c.restart, limit - total);
    int k = 0;
    for (int j = 0; j < mres; ++j) {
      bool replayed = false;
      if (graph && !(direct_first && j == 0)) {
        if (!p->garn[j])
          p->garn[j] = capture_launches(p, Bt, [&](const Batch& Bc) { return arnoldi_launches(p, Bc, c, j); },
                                        &p->garn_launches[j]);
        if (p->garn[j]) {
          CK(cudaGraphLaunch(p->garn[j], p->stream));
          p->launches += p->garn_launches[j];
          p->prec_applies += 1;
          p->matvecs += 1;
          replayed = true;
        }
      }
      if (!replayed && (rc = arnoldi_launches(p, Bt, c, j))) return rc;
      direct_first = false;
      if ((rc = read_scal(B, hs, 1))) return rc;
      k = j + 1;
      total += 1;
      if (hs->flags & 4) return PCB_ERR_NONFINITE;
      if (c.fixed <= 0 && (hs->flags & 1)) break;
      if (hs->flags & 8) break;
    }
    // x += Z y
    CK(LC(p) launch_multiaxpy(B, SL_ZBASE, k - 1, s_x, -1));
    CK(cudaMemsetAsync(&p->dSc->flags, 0, sizeof(int), p->stream));
    *it_out = total;
    if (c.fixed <= 0 && (hs->flags & 1)) {
      if (!c.check_true) { *relres_out = hs->est; return PCB_OK; }   // inner solve: as for MINRES
      CK(P_matvec(p, B, op, s_x, SL_R, s_b, EPI_RESID));
      CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
      if ((rc = read_scal(B, hs, 1))) return rc;
      *relres_out = std::sqrt(hs->dot1) / hs->bnorm;
      if (*relres_out <= c.tol) { *conv_out = true; return PCB_OK; }
    }
  }
  if (!c.check_true) { *relres_out = hs->est; return PCB_OK; }
  CK(P_matvec(p, B, op, s_x, SL_R, s_b, EPI_RESID));
  CK(LC(p) launch_reduce(B, B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
  if ((rc = read_scal(B, hs, 1))) return rc;
  *relres_out = std::sqrt(hs->dot1) / hs->bnorm;
  *conv_out = *relres_out <= c.tol;
  return PCB_OK;
}

static void resolve_defaults(const pcb_problem* p, const pcb_solve_opts* o, SolveCfg& c) {
  c.method = o ? o->method : PCB_METHOD_AUTO;
  c.kind = o ? o->precond : PCB_PREC_NONE;
  c.tol = (o && o->tol > 0) ? o->tol : 1e-8;
  c.maxit = (o && o->maxit > 0) ? o->maxit : 500;
  c.restart = (o && o->restart > 0) ? std::min(o->restart, PCB_MAX_RESTART) : 30;
  c.fixed = o ? o->fixed_iterations : 0;
  c.prec = p->desc.precision;
  c.inner_floor = (o && o->inner_floor > 0) ? o->inner_floor : 0.0;
  c.graphs = !(o && o->no_graphs);
  const bool va = p->g.mg_route != 0;
  if (c.method == PCB_METHOD_AUTO) {
    if (p->g.theta == 1.0 && p->g.bc != PCB_BC_NEUMANN) c.method = PCB_MINRES;
    else c.method = va ? PCB_FGMRES : PCB_GMRES;
    if (c.kind == PCB_PREC_NONE) {
      if (c.method == PCB_MINRES) c.kind = va ? PCB_PREC_PMS : PCB_PREC_ABS_PS;
      else c.kind = PCB_PREC_PS;
    }
  }
  c.op = c.method == PCB_MINRES ? PCB_OP_A : PCB_OP_AHAT;
}

static int solve_impl(pcb_problem* p, const pcb_solve_opts* o, const double* b_dev, double* x_dev,
                      pcb_solve_info* info) {
  SolveCfg c;
  resolve_defaults(p, o, c);
  if (c.method == PCB_MINRES && (c.kind == PCB_PREC_PS)) return PCB_ERR_INVALID_ARG;   // P_S is not SPD
  if (c.kind == PCB_PREC_ABS_PS && p->g.mg_route) return PCB_ERR_UNSUPPORTED;
  if (p->g.bc == PCB_BC_NEUMANN && (c.method == PCB_MINRES || c.kind != PCB_PREC_PS)) return PCB_ERR_UNSUPPORTED;
  int rc;
  if ((rc = ensure_minres(p))) return rc;
  const size_t nv = (size_t)2 * p->g.mn;
  double* v = p->vec_minres;
  p->hS.v[SL_R1] = v + 0 * nv; p->hS.v[SL_R2] = v + 1 * nv; p->hS.v[SL_Y] = v + 2 * nv; p->hS.v[SL_YO] = v + 3 * nv;
  p->hS.v[SL_Q] = v + 4 * nv; p->hS.v[SL_W] = v + 5 * nv; p->hS.v[SL_W2] = v + 6 * nv;
  p->hS.v[SL_R] = v + 0 * nv;
  if (c.method != PCB_MINRES) {
    if ((rc = ensure_gmres(p, c.restart))) return rc;
    p->hS.v[SL_VBASE] = p->vec_gmres;
    p->hS.v[SL_ZBASE] = p->vec_gmres + (size_t)(c.restart + 1) * nv;
  }
  p->hS.v[SL_X] = x_dev;
  p->hS.v[SL_B] = (double*)b_dev;
  const bool mixed = c.prec == PCB_MIXED;
  if (mixed) {
    if ((rc = ensure_mixed(p))) return rc;
    p->hS.v[SL_BI] = p->vec_mixed;
    p->hS.v[SL_XI] = p->vec_mixed + nv;
  }
  if ((rc = upload_slots(p))) return rc;
  Scal* hs = p->hSc;
  p->launches = 0; p->prec_applies = 0; p->matvecs = 0; p->matvecs_inner = 0;
  p->prof = o && o->profile;
  p->ev_prec_used = 0; p->ev_mv_used = 0; p->ev_mvi_used = 0;
  auto t0 = std::chrono::steady_clock::now();
  int iters = 0, sweeps = 0;
  double relres = 1.0;
  bool conv = false;
  auto run = [&](SolveCfg& cc, int sb, int sx, double* rel, int* it, bool* cv) {
    return cc.method == PCB_MINRES ? minres_single(p, cc, sb, sx, hs, rel, it, cv)
                                   : fgmres_single(p, cc, sb, sx, hs, rel, it, cv);
  };
  if (!mixed) {
    c.check_true = true;
    rc = run(c, SL_B, SL_X, &relres, &iters, &conv);
    sweeps = 1;
  } else {
    // FP64 iterative refinement around the FP32-preconditioned inner solve:
    //   r = b - op x ; solve op d = r (inner tolerance tol*||b||/||r||) ; x += d
    const int max_ref = (o && o->max_refinements > 0) ? o->max_refinements : 10;
    const size_t vbytes = nv * sizeof(double);
    CK(cudaMemsetAsync(x_dev, 0, vbytes, p->stream));
    CK(LC(p) launch_dot(p->B, SL_B, SL_B));
    CK(LC(p) launch_reduce(p->B, p->B.off_vec, 1, 0, SS_BNORM, c.tol, 0, 0));
    if ((rc = read_scal(p->B, hs, 1))) return rc;
    const double bnorm = hs->bnorm;
    if (!std::isfinite(bnorm)) return PCB_ERR_NONFINITE;
    CK(LC(p) launch_axpby(p->B, AX_COPY, SL_B, SL_BI, -1));
    double rnorm = bnorm;
    rc = PCB_OK;
    if (bnorm == 0.0) { conv = true; relres = 0.0; }
    while (!conv && sweeps < max_ref && iters < c.maxit) {
      SolveCfg ci = c;
      ci.check_true = false;
      ci.tol = std::min(0.5, std::max(c.tol * bnorm / rnorm, c.inner_floor));
      ci.maxit = c.maxit - iters;
      double rel_in; int it_in; bool cv_in;
      rc = run(ci, SL_BI, SL_XI, &rel_in, &it_in, &cv_in);
      if (rc) break;
      iters += it_in;
      sweeps += 1;
      // x += d ; r = b - op x  (into the inner right-hand side slot)
      CK(LC(p) launch_axpby(p->B, AX_ADD, SL_XI, SL_X, -1));
      CK(P_matvec(p, p->B, c.op, SL_X, SL_BI, SL_B, EPI_RESID));
      CK(LC(p) launch_reduce(p->B, p->B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
      if ((rc = read_scal(p->B, hs, 1))) break;
      rnorm = std::sqrt(hs->dot1);
      relres = rnorm / bnorm;
      if (!std::isfinite(relres)) { rc = PCB_ERR_NONFINITE; break; }
      if (relres <= c.tol) conv = true;
      if (c.fixed > 0) break;
    }
  }
  CK(cudaStreamSynchronize(p->stream));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == PCB_OK && !conv && c.fixed <= 0) rc = PCB_NOT_CONVERGED;
  if (info) {
    info->status = rc; info->method = c.method; info->precond = c.kind; info->iterations = iters;
    info->refinements = sweeps; info->relres = relres; info->seconds = secs;
    info->launches = p->launches; info->precond_applies = p->prec_applies; info->matvecs = p->matvecs;
    info->precond_ms = p->prof ? ev_sum(p->ev_prec, p->ev_prec_used) : 0.0;
    info->matvec_ms = p->prof ? ev_sum(p->ev_mv, p->ev_mv_used) + ev_sum(p->ev_mvi, p->ev_mvi_used) : 0.0;
    info->matvecs_inner = p->matvecs_inner;
    info->matvec_inner_ms = p->prof ? ev_sum(p->ev_mvi, p->ev_mvi_used) : 0.0;
  }
  return rc;
}

extern "C" {

int pcb_assemble_rhs(pcb_problem* p, int op, const double* g_dev, const double* f_dev, const double* y0_dev,
                     double* b_dev) {
  if (!p || !g_dev || !f_dev || !b_dev || (op != PCB_OP_A && op != PCB_OP_AHAT)) return PCB_ERR_INVALID_ARG;
  if (p->g.fem && y0_dev) return PCB_ERR_UNSUPPORTED;
  CK(launch_rhs(p->g, p->stream, op, g_dev, f_dev, y0_dev, b_dev));
  if (p->g.fem) {
    // f~, g~ carry M (Sec. 1) and the system's right-hand side M^{-1/2}: with y0 = 0 both halves are
    // M^{1/2} applied to the time combinations of the samples (FEM_MASS_SQRT = 0)
    p->hS.v[SL_UIN] = b_dev;
    p->hS.v[SL_UOUT] = b_dev;
    int rc;
    if ((rc = upload_slots(p))) return rc;
    CK(launch_fem_spatial(p->B, 0, PCB_OP_A, SL_UIN, SL_UOUT));
  }
  return PCB_OK;
}

int pcb_matvec(pcb_problem* p, int op, const double* x_dev, double* y_dev) {
  if (!p || !x_dev || !y_dev || (op != PCB_OP_A && op != PCB_OP_AHAT)) return PCB_ERR_INVALID_ARG;
  if (x_dev == y_dev) return PCB_ERR_INVALID_ARG;
  p->hS.v[SL_UIN] = (double*)x_dev;
  p->hS.v[SL_UOUT] = y_dev;
  int rc;
  if ((rc = upload_slots(p))) return rc;
  CK(launch_matvec(p->B, op, SL_UIN, SL_UOUT, -1, EPI_PLAIN));
  return PCB_OK;
}

int pcb_lanczos_product(pcb_problem* p, int precision, const double* y_dev, const double* r1_dev, double beta,
                        double oldb, double* out_dev, double* dot) {
  if (!p || !y_dev || !out_dev || !dot) return PCB_ERR_INVALID_ARG;
  if (precision != PCB_FP64 && precision != PCB_MIXED) return PCB_ERR_INVALID_ARG;
  if (!(beta > 0.0) || !std::isfinite(beta) || !(oldb >= 0.0) || !std::isfinite(oldb)) return PCB_ERR_INVALID_ARG;
  if ((oldb > 0.0 && !r1_dev) || out_dev == y_dev || (r1_dev && out_dev == r1_dev)) return PCB_ERR_INVALID_ARG;
  Scal* hs = p->hSc;
  CK(cudaStreamSynchronize(p->stream));   // the pinned scalar buffer may still be in flight
  std::memset(hs, 0, sizeof(Scal));
  hs->beta = beta;
  hs->oldb = oldb;
  hs->itn = oldb > 0.0 ? 1 : 0;
  hs->active = 1;
  CK(cudaMemcpyAsync(p->dSc, hs, sizeof(Scal), cudaMemcpyHostToDevice, p->stream));
  p->hS.v[SL_UIN] = (double*)y_dev;
  p->hS.v[SL_UOUT] = out_dev;
  p->hS.v[SL_UAUX] = (double*)r1_dev;
  int rc;
  if ((rc = upload_slots(p))) return rc;
  const int epi = EPI_MINRES | (precision == PCB_MIXED ? EPI_FAST : 0);
  CK(launch_matvec(p->B, PCB_OP_A, SL_UIN, SL_UOUT, oldb > 0.0 ? SL_UAUX : -1, epi));
  CK(launch_reduce(p->B, p->B.off_mv, 1, 0, SS_NORM, 0.0, 0, 0));
  if ((rc = read_scal(p->B, hs, 1))) return rc;
  *dot = hs->dot1;
  return PCB_OK;
}

int pcb_precond_apply(pcb_problem* p, int kind, int precision, const double* x_dev, double* y_dev) {
  if (!p || !x_dev || !y_dev) return PCB_ERR_INVALID_ARG;
  if (kind != PCB_PREC_ABS_PS && kind != PCB_PREC_PS && kind != PCB_PREC_PMS) return PCB_ERR_INVALID_ARG;
  if (precision != PCB_FP64 && precision != PCB_MIXED) return PCB_ERR_INVALID_ARG;
  if (kind == PCB_PREC_ABS_PS && p->g.mg_route) return PCB_ERR_UNSUPPORTED;
  if (kind != PCB_PREC_PS && p->g.bc == PCB_BC_NEUMANN) return PCB_ERR_UNSUPPORTED;
  p->hS.v[SL_UIN] = (double*)x_dev;
  p->hS.v[SL_UOUT] = y_dev;
  int rc;
  if ((rc = upload_slots(p))) return rc;
  return apply_precond(p, p->B, kind, precision, SL_UIN, SL_UOUT);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Autotuner (pcb_autotune): times the preconditioner apply of one problem under each candidate
// kernel configuration and keeps the fastest.  Candidates (constant coefficient only):
//   * the pipelined FP32 kernel families on or off for the spatial and the time passes, and the
//     n = 512 time-major hand-off on or off;
//   * for the tile kernels, the register-FFT radix (values per lane Q, i.e. P = M / Q lanes per
//     line, with Q and 2Q where the kernels support them) and the tile size (lines or columns
//     per block, from a per-tile element budget at 1/2, 1 and 2 times the default).
// ---------------------------------------------------------------------------------------------
namespace {

__global__ void k_tune_fill(double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = sin(0.37 * (double)(i % 100003)) + 0.25;
}

// out[0] = max |a - b|, out[1] = max |b| (non-negative doubles order like their bit patterns, so
// an integer atomic max serves; out must start at zero)
__global__ void k_tune_diff(const double* __restrict__ a, const double* __restrict__ b, long long n,
                            unsigned long long* __restrict__ out) {
  double d = 0.0, r = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double bi = b[i];
    d = fmax(d, fabs(a[i] - bi));
    r = fmax(r, fabs(bi));
  }
  if (!(d == d)) d = INFINITY;      // a NaN difference counts as infinite
  for (int o = 16; o > 0; o >>= 1) {
    d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
    r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(out, (unsigned long long)__double_as_longlong(d));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(r));
  }
}

constexpr size_t kSmemMax = 227 * 1024;

double __longlong_as_double_host(unsigned long long v) {
  double d;
  std::memcpy(&d, &v, sizeof(d));
  return d;
}

bool tune_valid(const Geom& g0, TuneChoice c, int prec) {
  Geom g = g0;
  apply_choice(g, c);
  const int pr = prec == PCB_MIXED ? 1 : 0;
  const bool pipe_d = pr && pipe_dst_p(g), pipe_t = pr && pipe_time_p(g);
  if (!pipe_d && dst_smem_bytes(g, pr) > kSmemMax) return false;
  if (!pipe_t && time_smem_bytes(g, pr) > kSmemMax) return false;
  return true;
}

std::vector<TuneChoice> tune_candidates(const Geom& g, int prec) {
  const int q0d = dst_Q(g.M), q0t = time_Q(g.n);
  std::vector<int> qd{q0d}, qt{q0t};
  const int P0d = g.M / q0d;
  if (2 * q0d <= 24 && q_supported(2 * q0d) && P0d >= 2 && g.M % (2 * q0d) == 0) qd.push_back(2 * q0d);
  if (2 * q0t <= 16 && g.n / q0t >= 2) qt.push_back(2 * q0t);
  std::vector<TuneChoice> out;
  auto add = [&](int tune, int dq, int tq) {
    const TuneChoice c{tune, dq, tq};
    for (const auto& o : out) if (o.tune == c.tune && o.dst_q == dq && o.time_q == tq) return;
    if (tune_valid(g, c, prec)) out.push_back(c);
  };
  add(0, q0d, q0t);                                   // the default shapes come first
  Geom d = g;
  apply_choice(d, out.empty() ? TuneChoice{0, q0d, q0t} : out[0]);
  const bool mixed = prec == PCB_MIXED;
  const bool can_pipe_t = mixed && pipe_time_p(d), can_pipe_d = mixed && pipe_dst_p(d);
  if (can_pipe_d && can_pipe_t && g.n == 512) add(TUNE_NO_HANDOFF, q0d, q0t);
  if (can_pipe_t && g.n == 512 && g.zeta_pi) {
    for (int v : {TUNE_TIME512_3BLK, TUNE_TIME512_4BLK}) {
      add(v, q0d, q0t);
      if (can_pipe_d) add(v | TUNE_NO_HANDOFF, q0d, q0t);
    }
  }
  for (int b = 0; b < 3; ++b) {
    const int bs = b << 4;
    for (int dq : qd) {
      if (can_pipe_t) add(TUNE_NO_PIPE_DST | bs, dq, q0t);          // tile spatial passes, pipelined time
      for (int tq : qt) add(TUNE_NO_PIPE_DST | TUNE_NO_PIPE_TIME | bs, dq, tq);   // tile kernels only
    }
  }
  return out;
}

// the configuration a problem runs, in the terms of pcb_tune_info
void describe_choice(const Geom& g, int prec, pcb_tune_info* info) {
  info->pipelined_dst = prec == PCB_MIXED && pipe_dst_p(g);
  info->pipelined_time = prec == PCB_MIXED && pipe_time_p(g);
  info->time_major_handoff = prec == PCB_MIXED && (pipe_dst_code(g) & 64) ? 1 : 0;
  info->dst_lanes = g.M / g.dst_q;
  info->time_lanes = g.n / g.time_q;
  info->tile_scale = tune_budget_shift(g.tune) == 1 ? 0.5 : tune_budget_shift(g.tune) == 2 ? 2.0 : 1.0;
  info->time512_blocks = (g.tune & TUNE_TIME512_3BLK) ? 3 : (g.tune & TUNE_TIME512_4BLK) ? 4 : 2;
}

}  // namespace

extern "C" {

int pcb_autotune(pcb_problem* p, int kind, int reps, pcb_tune_info* info) {
  if (!p) return PCB_ERR_INVALID_ARG;
  if (kind == PCB_PREC_NONE) kind = p->g.bc == PCB_BC_NEUMANN ? PCB_PREC_PS : PCB_PREC_ABS_PS;
  if (kind != PCB_PREC_ABS_PS && kind != PCB_PREC_PS && kind != PCB_PREC_PMS) return PCB_ERR_INVALID_ARG;
  if (p->g.mg_route) return PCB_ERR_UNSUPPORTED;     // the multigrid route is not tuned
  if (kind != PCB_PREC_PS && p->g.bc == PCB_BC_NEUMANN) return PCB_ERR_UNSUPPORTED;
  if (reps <= 0) reps = 3;
  const int prec = p->desc.precision;
  const size_t nv = (size_t)2 * p->g.mn;
  double* buf = nullptr;
  unsigned long long* dmax = nullptr;
  unsigned long long hmax[2] = {0, 0};
  if (cudaMalloc(&buf, 3 * nv * sizeof(double)) != cudaSuccess || cudaMalloc(&dmax, 2 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError(); cudaFree(buf); return PCB_ERR_OUT_OF_MEMORY;
  }
  auto done = [&](int rc) { cudaStreamSynchronize(p->stream); cudaFree(buf); cudaFree(dmax); return rc; };
  double* yref = buf + 2 * nv;
  // a candidate whose result differs from the default configuration's by more than the rounding of
  // the precision (relative max-norm) is rejected rather than timed
  const double vtol = prec == PCB_MIXED ? 1e-5 : 1e-12;
  int rejected = 0;
  k_tune_fill<<<1024, 256, 0, p->stream>>>(buf, (long long)nv);
  p->hS.v[SL_UIN] = buf;
  p->hS.v[SL_UOUT] = buf + nv;
  int rc;
  if ((rc = upload_slots(p))) return done(rc);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return done(PCB_ERR_CUDA);
  const Geom g0 = p->g;
  Geom gd = g0;
  gd.tune = 0; gd.dst_q = dst_Q(gd.M); gd.time_q = time_Q(gd.n);
  set_shapes(gd);
  const std::vector<TuneChoice> cands = tune_candidates(gd, prec);
  std::vector<int> staging;
  // make candidate c the problem's configuration (host mirror, device Geom, launch offsets)
  auto install = [&](const TuneChoice& c) -> int {
    Geom g = gd;
    apply_choice(g, c);
    g.scratch = g0.scratch;
    p->g = g;
    CK(cudaMemcpyAsync(p->dG, &p->g, sizeof(Geom), cudaMemcpyHostToDevice, p->stream));
    int r = fill_batch(p->B, std::vector<Geom>(1, p->g), p->doff, p->stream, staging);
    if (r) return r;
    CK(cudaStreamSynchronize(p->stream));
    return PCB_OK;
  };
  double best = 1e300, def_ms = 0.0;
  int best_k = -1, timed = 0;
  for (size_t k = 0; k < cands.size(); ++k) {
    if ((rc = install(cands[k]))) break;
    if (launch_precond_fast(p->B, kind, prec, SL_UIN, SL_UOUT) != cudaSuccess) { cudaGetLastError(); continue; }
    if (k == 0) {
      if (cudaMemcpyAsync(yref, buf + nv, nv * sizeof(double), cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess) {
        cudaGetLastError(); break;
      }
    } else {
      if (cudaMemsetAsync(dmax, 0, 2 * sizeof(unsigned long long), p->stream) != cudaSuccess) { cudaGetLastError(); break; }
      k_tune_diff<<<1024, 256, 0, p->stream>>>(buf + nv, yref, (long long)nv, dmax);
      if (cudaMemcpyAsync(hmax, dmax, sizeof(hmax), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
          cudaStreamSynchronize(p->stream) != cudaSuccess) { cudaGetLastError(); break; }
      const double dm = __longlong_as_double_host(hmax[0]), rm = __longlong_as_double_host(hmax[1]);
      if (!(dm <= vtol * rm)) { ++rejected; continue; }
    }
    cudaEventRecord(e0, p->stream);
    bool ok = true;
    for (int r = 0; r < reps && ok; ++r) ok = launch_precond_fast(p->B, kind, prec, SL_UIN, SL_UOUT) == cudaSuccess;
    cudaEventRecord(e1, p->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess || !ok) { cudaGetLastError(); continue; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double avg = ms / reps;
    ++timed;
    if (k == 0) def_ms = avg;
    if (avg < best) { best = avg; best_k = (int)k; }
  }
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  if (best_k < 0) {           // nothing could be timed: keep the configuration the problem had
    p->g = g0;
    cudaMemcpyAsync(p->dG, &p->g, sizeof(Geom), cudaMemcpyHostToDevice, p->stream);
    fill_batch(p->B, std::vector<Geom>(1, p->g), p->doff, p->stream, staging);
    return done(rc ? rc : PCB_ERR_CUDA);
  }
  if ((rc = install(cands[best_k]))) return done(rc);
  // captured iterations launch the kernels of the old configuration
  if (p->git) { cudaGraphExecDestroy(p->git); p->git = nullptr; }
  for (cudaGraphExec_t& e : p->garn) if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  p->git_kind = p->garn_kind = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[tune_key(p->g, prec)] = cands[best_k];
  }
  if (info) {
    describe_choice(p->g, prec, info);
    info->candidates = timed;
    info->rejected = rejected;
    info->chosen = best_k;
    info->default_ms = def_ms;
    info->best_ms = best;
  }
  return done(PCB_OK);
}

int pcb_tune_select(pcb_problem* p, int candidate, pcb_tune_info* info) {
  if (!p) return PCB_ERR_INVALID_ARG;
  if (p->g.mg_route) return PCB_ERR_UNSUPPORTED;
  const int prec = p->desc.precision;
  Geom gd = p->g;
  gd.tune = 0; gd.dst_q = dst_Q(gd.M); gd.time_q = time_Q(gd.n);
  set_shapes(gd);
  const std::vector<TuneChoice> cands = tune_candidates(gd, prec);
  if (candidate >= (int)cands.size()) return PCB_ERR_INVALID_ARG;
  if (candidate >= 0) {
    CK(cudaStreamSynchronize(p->stream));
    Geom g = gd;
    apply_choice(g, cands[candidate]);
    g.scratch = p->g.scratch;
    p->g = g;
    CK(cudaMemcpyAsync(p->dG, &p->g, sizeof(Geom), cudaMemcpyHostToDevice, p->stream));
    std::vector<int> staging;
    int rc = fill_batch(p->B, std::vector<Geom>(1, p->g), p->doff, p->stream, staging);
    if (rc) return rc;
    CK(cudaStreamSynchronize(p->stream));
    if (p->git) { cudaGraphExecDestroy(p->git); p->git = nullptr; }
    for (cudaGraphExec_t& e : p->garn) if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    p->git_kind = p->garn_kind = -1;
  }
  if (info) {
    describe_choice(p->g, prec, info);
    info->candidates = (int)cands.size();
    info->rejected = 0;
    info->chosen = candidate;
    info->default_ms = info->best_ms = 0.0;
  }
  return PCB_OK;
}

int pcb_recover(pcb_problem* p, const double* x_dev, double* y_dev, double* p_dev) {
  if (!p || !x_dev || !y_dev || !p_dev) return PCB_ERR_INVALID_ARG;
  if (p->g.fem) {
    // (B2^{-1} (x) M^{-1/2}): the spatial factor first (FEM_MASS_ISQRT = 1) into a staging vector
    const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
    if (!p->host_io) {
      if (cudaMalloc(&p->host_io, 2 * vb) != cudaSuccess) { cudaGetLastError(); p->host_io = nullptr; return PCB_ERR_OUT_OF_MEMORY; }
      p->bytes += 2 * vb;
    }
    p->hS.v[SL_UIN] = (double*)x_dev;
    p->hS.v[SL_UOUT] = p->host_io;
    int rc;
    if ((rc = upload_slots(p))) return rc;
    CK(launch_fem_spatial(p->B, 1, PCB_OP_A, SL_UIN, SL_UOUT));
    CK(launch_recover(p->g, p->stream, p->host_io, y_dev, p_dev));
    return PCB_OK;
  }
  CK(launch_recover(p->g, p->stream, x_dev, y_dev, p_dev));
  return PCB_OK;
}

int pcb_solve(pcb_problem* p, const pcb_solve_opts* o, const double* b_dev, double* x_dev, pcb_solve_info* info) {
  if (!p || !b_dev || !x_dev || b_dev == x_dev) return PCB_ERR_INVALID_ARG;
  return solve_impl(p, o, b_dev, x_dev, info);
}

int pcb_solve_host(pcb_problem* p, const pcb_solve_opts* o, const double* b_host, double* x_host,
                   pcb_solve_info* info) {
  if (!p || !b_host || !x_host) return PCB_ERR_INVALID_ARG;
  const size_t vb = (size_t)2 * p->g.mn * sizeof(double);
  if (!p->host_io) {
    if (cudaMalloc(&p->host_io, 2 * vb) != cudaSuccess) { cudaGetLastError(); p->host_io = nullptr; return PCB_ERR_OUT_OF_MEMORY; }
    p->bytes += 2 * vb;
  }
  double* b = p->host_io;
  double* x = p->host_io + 2 * p->g.mn;
  int rc = PCB_OK;
  // page-locked buffers move with a copy kernel, pageable ones with the runtime's copy
  long long copies = 0;
  if (copy_host(b, b_host, 2 * p->g.mn, true, p->stream, &copies) != cudaSuccess) rc = PCB_ERR_CUDA;
  if (rc == PCB_OK) rc = solve_impl(p, o, b, x, info);
  if ((rc == PCB_OK || rc == PCB_NOT_CONVERGED) &&
      copy_host(x_host, x, 2 * p->g.mn, false, p->stream, &copies) != cudaSuccess)
    rc = PCB_ERR_CUDA;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess && rc == PCB_OK) rc = PCB_ERR_CUDA;
  if (info) info->launches += copies;
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batched solves: instances of any size share every launch.  Instances are grouped by method
// (MINRES for the symmetric system, (F)GMRES otherwise); each group iterates in lockstep and
// instances leave through the device-side `active` mask when their inner solve ends.  Every
// instance runs rounds of: inner Krylov solve from a zero guess on r = b - op x to the tolerance
// tol*||b||/||r|| (recurrence estimate), then x += d and the FP64 true residual.  With FP64 the
// first round normally finishes; with the FP32 preconditioner later rounds are the refinement.
// ---------------------------------------------------------------------------------------------
namespace {

struct BGroup {
  std::vector<pcb_problem*> probs;
  std::vector<int> idx;               // positions in the caller's arrays
  int method = PCB_MINRES, op = PCB_OP_A, kind = PCB_PREC_ABS_PS, prec = PCB_MIXED;
  Batch B;
  Geom* dG = nullptr; Slots* dS = nullptr; Scal* dSc = nullptr; int* dAct = nullptr; int* dOff = nullptr;
  double* dPart = nullptr; double* dTol = nullptr;
  Scal* hSc = nullptr; int* hAct = nullptr; double* hTol = nullptr;
  std::vector<double> bnorm, rnorm;
  std::vector<int> iters, sweeps, status, done, in_round, round_member;
  int j = 0;                          // Arnoldi index (lockstep)
  int it_round = 0;
  bool round_open = false;
  // Lockstep iterations replayed from CUDA graphs: the group's launches take their instances,
  // slot pointers, masks and tolerances from device memory, so one capture serves every round
  // (MINRES) or every round at one Arnoldi index (FGMRES).  The first iteration runs directly.
  cudaStream_t cap = nullptr;
  cudaGraphExec_t git = nullptr;
  std::vector<cudaGraphExec_t> garn;
  int direct = 0;                     // iterations launched directly so far
  ~BGroup() {
    if (git) cudaGraphExecDestroy(git);
    for (cudaGraphExec_t e : garn) if (e) cudaGraphExecDestroy(e);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(dG); cudaFree(dS); cudaFree(dSc); cudaFree(dAct); cudaFree(dOff); cudaFree(dPart); cudaFree(dTol);
    cudaFreeHost(hSc); cudaFreeHost(hAct); cudaFreeHost(hTol);
  }
};

// capture the launches issue(Bc) makes into an executable graph, on the group's private stream
// (the group's own may be the legacy default stream); null when capture is not possible
template <typename F>
static cudaGraphExec_t capture_group(BGroup& G, F&& issue) {
  if (!G.cap && cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError(); G.cap = nullptr; return nullptr;
  }
  Batch Bc = G.B;
  Bc.stream = G.cap;
  if (cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  const int rc = issue(Bc);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(G.cap, &graph);
  if (rc != PCB_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return exec;
}

int set_active(BGroup& G, const std::vector<int>& mask) {
  const int n = (int)G.probs.size();
  CK(cudaStreamSynchronize(G.B.stream));
  for (int k = 0; k < n; ++k) G.hAct[k] = mask[k];
  CK(cudaMemcpyAsync(G.dAct, G.hAct, n * sizeof(int), cudaMemcpyHostToDevice, G.B.stream));
  return PCB_OK;
}

int read_all(BGroup& G) {
  CK(cudaMemcpyAsync(G.hSc, G.dSc, sizeof(Scal) * G.probs.size(), cudaMemcpyDeviceToHost, G.B.stream));
  CK(cudaStreamSynchronize(G.B.stream));
  return PCB_OK;
}

int group_setup(BGroup& G, const SolveCfg& c, const double* const* b_dev, double* const* x_dev, cudaStream_t st) {
  const int n = (int)G.probs.size();
  std::vector<Geom> gs;
  std::vector<Slots> sl(n);
  for (int k = 0; k < n; ++k) {
    pcb_problem* p = G.probs[k];
    int rc;
    if ((rc = ensure_minres(p)) || (rc = ensure_mixed(p))) return rc;
    if (G.method != PCB_MINRES && (rc = ensure_gmres(p, c.restart))) return rc;
    const size_t nv = (size_t)2 * p->g.mn;
    double* v = p->vec_minres;
    Slots& S = sl[k];
    std::memset(&S, 0, sizeof(S));
    S.v[SL_R1] = v; S.v[SL_R2] = v + nv; S.v[SL_Y] = v + 2 * nv; S.v[SL_YO] = v + 3 * nv; S.v[SL_Q] = v + 4 * nv;
    S.v[SL_W] = v + 5 * nv; S.v[SL_W2] = v + 6 * nv; S.v[SL_R] = v;
    S.v[SL_BI] = p->vec_mixed; S.v[SL_XI] = p->vec_mixed + nv;
    if (G.method != PCB_MINRES) { S.v[SL_VBASE] = p->vec_gmres; S.v[SL_ZBASE] = p->vec_gmres + (size_t)(c.restart + 1) * nv; }
    S.v[SL_X] = x_dev[G.idx[k]];
    S.v[SL_B] = (double*)b_dev[G.idx[k]];
    gs.push_back(p->g);
  }
  size_t part = 0; int tv = 0, tm = 0;
  for (const Geom& g : gs) { tv += g.vec_blocks; tm += g.mv_blocks; }
  part = std::max((size_t)tv * (PCB_MAX_RESTART + 1), (size_t)tm) + 1;
  if (cudaMalloc(&G.dG, sizeof(Geom) * n) || cudaMalloc(&G.dS, sizeof(Slots) * n) ||
      cudaMalloc(&G.dSc, sizeof(Scal) * n) || cudaMalloc(&G.dAct, sizeof(int) * n) ||
      cudaMalloc(&G.dOff, sizeof(int) * 10 * (n + 1)) || cudaMalloc(&G.dPart, part * sizeof(double)) ||
      cudaMalloc(&G.dTol, sizeof(double) * n) || cudaMallocHost(&G.hSc, sizeof(Scal) * n) ||
      cudaMallocHost(&G.hAct, sizeof(int) * n) || cudaMallocHost(&G.hTol, sizeof(double) * n)) {
    cudaGetLastError();
    return PCB_ERR_OUT_OF_MEMORY;
  }
  CK(cudaMemcpyAsync(G.dG, gs.data(), sizeof(Geom) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(G.dS, sl.data(), sizeof(Slots) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(G.dSc, 0, sizeof(Scal) * n, st));
  std::vector<int> staging;
  std::memset(&G.B, 0, sizeof(Batch));
  int rc = fill_batch(G.B, gs, G.dOff, st, staging);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st));
  G.B.G = G.dG; G.B.S = G.dS; G.B.Sc = G.dSc; G.B.active = G.dAct; G.B.partial = G.dPart; G.B.tols = G.dTol;
  G.bnorm.assign(n, 0.0); G.rnorm.assign(n, 0.0); G.iters.assign(n, 0); G.sweeps.assign(n, 0);
  G.status.assign(n, PCB_OK); G.done.assign(n, 0); G.in_round.assign(n, 0); G.round_member.assign(n, 0);
  // ||b|| for every instance; x = 0; inner right-hand side = b
  std::vector<int> all(n, 1);
  if ((rc = set_active(G, all))) return rc;
  CK(launch_axpby(G.B, AX_ZERO, -1, SL_X, -1));
  CK(launch_axpby(G.B, AX_COPY, SL_B, SL_BI, -1));
  CK(launch_dot(G.B, SL_B, SL_B));
  CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_BNORM, c.tol, 0, 0));
  if ((rc = read_all(G))) return rc;
  for (int k = 0; k < n; ++k) {
    G.bnorm[k] = G.hSc[k].bnorm; G.rnorm[k] = G.bnorm[k];
    if (!std::isfinite(G.bnorm[k])) { G.status[k] = PCB_ERR_NONFINITE; G.done[k] = 1; }
    else if (G.bnorm[k] == 0.0) { G.done[k] = 1; G.rnorm[k] = 0.0; }
  }
  return PCB_OK;
}

// start a round for every unfinished instance
int round_start(BGroup& G, const SolveCfg& c) {
  const int n = (int)G.probs.size();
  std::vector<int> mask(n, 0);
  int any = 0;
  for (int k = 0; k < n; ++k) {
    if (G.done[k]) continue;
    mask[k] = 1; any = 1;
    G.hTol[k] = std::min(0.5, std::max(c.tol * G.bnorm[k] / G.rnorm[k], c.inner_floor));
  }
  G.round_member = mask; G.in_round = mask; G.round_open = any; G.it_round = 0; G.j = 0;
  if (!any) return PCB_OK;
  int rc;
  if ((rc = set_active(G, mask))) return rc;
  CK(cudaMemcpyAsync(G.dTol, G.hTol, sizeof(double) * n, cudaMemcpyHostToDevice, G.B.stream));
  CK(launch_axpby(G.B, AX_ZERO, -1, SL_XI, -1));
  if (G.method == PCB_MINRES) {
    CK(launch_axpby(G.B, AX_ZERO, -1, SL_W, -1));
    CK(launch_axpby(G.B, AX_ZERO, -1, SL_W2, -1));
    CK(launch_axpby(G.B, AX_COPY, SL_BI, SL_R1, -1));
    CK(launch_axpby(G.B, AX_COPY, SL_BI, SL_R2, -1));
    if ((rc = apply_precond(G.probs[0], G.B, G.kind, G.prec, SL_R2, SL_Y))) return rc;
    CK(launch_dot(G.B, SL_R2, SL_Y));
    CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_MINRES_INIT, c.tol, 0, 0));
  } else {
    CK(launch_dot(G.B, SL_BI, SL_BI));
    CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_BNORM, c.tol, 0, 0));
    CK(launch_dot(G.B, SL_BI, SL_BI));
    CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_GMRES_START, c.tol, 0, 0));
    CK(launch_setslot(G.B, SL_VJ, SL_VBASE, 0));
    CK(launch_axpby(G.B, AX_SCALE_INV_BETA, SL_BI, SL_VJ, -1));
  }
  if ((rc = read_all(G))) return rc;
  for (int k = 0; k < n; ++k) {
    if (!mask[k]) continue;
    if (G.hSc[k].flags & 4) { G.status[k] = PCB_ERR_NONFINITE; G.done[k] = 1; G.in_round[k] = 0; }
    else if (G.method == PCB_MINRES && (G.hSc[k].flags & 2)) { G.status[k] = PCB_ERR_BREAKDOWN; G.done[k] = 1; G.in_round[k] = 0; }
  }
  return set_active(G, G.in_round);
}

// one lockstep iteration of the group's active instances; ends instances whose estimate is met
int round_step(BGroup& G, const SolveCfg& c) {
  const int n = (int)G.probs.size();
  int rc;
  pcb_problem* p0 = G.probs[0];
  std::vector<int> ending(n, 0);
  bool any_end = false;
  if (G.method == PCB_MINRES) {
    auto iter = [&](const Batch& Bx) -> int {
      CK(launch_matvec(Bx, PCB_OP_A, SL_Y, SL_Q, SL_R1, EPI_MINRES | (G.prec == PCB_MIXED ? EPI_FAST : 0)));
      CK(launch_reduce(Bx, Bx.off_mv, 1, 0, SS_MINRES_ALFA, c.tol, 0, 0));
      CK(launch_axpby(Bx, AX_MINRES_R, SL_Q, SL_R2, SL_R1));
      int r;
      if ((r = apply_precond(p0, Bx, G.kind, G.prec, SL_R1, SL_YO))) return r;
      CK(launch_dot(Bx, SL_R1, SL_YO));
      CK(launch_reduce(Bx, Bx.off_vec, 1, 0, SS_MINRES_GIVENS, c.tol, 0, 0));
      CK(launch_minres_wx(Bx, SL_Y, SL_W, SL_W2, SL_XI));
      CK(launch_swap(Bx, SL_R1, SL_R2, SL_Y, SL_YO, SL_W, SL_W2));
      return PCB_OK;
    };
    if (c.graphs && G.direct > 0 && !G.git) G.git = capture_group(G, iter);
    if (c.graphs && G.git) {
      CK(cudaGraphLaunch(G.git, G.B.stream));
    } else {
      if ((rc = iter(G.B))) return rc;
      ++G.direct;
    }
    if ((rc = read_all(G))) return rc;
    G.it_round += 1;
    for (int k = 0; k < n; ++k) {
      if (!G.in_round[k]) continue;
      G.iters[k] += 1;
      const int f = G.hSc[k].flags;
      if (f & 4) { G.status[k] = PCB_ERR_NONFINITE; G.done[k] = 1; ending[k] = 1; }
      else if (f & 2) { G.status[k] = PCB_ERR_BREAKDOWN; G.done[k] = 1; ending[k] = 1; }
      else if ((f & 1) || G.iters[k] >= c.maxit) ending[k] = 1;
      any_end |= ending[k] != 0;
    }
  } else {
    const int j = G.j;
    auto step = [&](const Batch& Bx) -> int {
      CK(launch_setslot(Bx, SL_VJ, SL_VBASE, j));
      CK(launch_setslot(Bx, SL_ZJ, SL_ZBASE, j));
      CK(launch_setslot(Bx, SL_VJ1, SL_VBASE, j + 1));
      int r;
      if ((r = apply_precond(p0, Bx, G.kind, G.prec, SL_VJ, SL_ZJ))) return r;
      CK(launch_matvec(Bx, G.op, SL_ZJ, SL_VJ1, -1, EPI_PLAIN));
      for (int pass = 0; pass < 2; ++pass) {
        CK(launch_multidot(Bx, SL_VBASE, j, SL_VJ1));
        CK(launch_reduce_multi(Bx, j, pass));
        CK(launch_multiaxpy(Bx, SL_VBASE, j, SL_VJ1, pass));
      }
      CK(launch_dot(Bx, SL_VJ1, SL_VJ1));
      CK(launch_reduce(Bx, Bx.off_vec, 1, 0, SS_GMRES_ARNOLDI, c.tol, j, c.restart));
      CK(launch_axpby(Bx, AX_SCALE_INV_HNORM, SL_VJ1, SL_VJ1, -1));
      return PCB_OK;
    };
    if ((int)G.garn.size() < c.restart) G.garn.resize(c.restart, nullptr);
    if (c.graphs && G.direct > 0 && !G.garn[j]) G.garn[j] = capture_group(G, step);
    if (c.graphs && G.garn[j]) {
      CK(cudaGraphLaunch(G.garn[j], G.B.stream));
    } else {
      if ((rc = step(G.B))) return rc;
      ++G.direct;
    }
    if ((rc = read_all(G))) return rc;
    G.it_round += 1;
    for (int k = 0; k < n; ++k) {
      if (!G.in_round[k]) continue;
      G.iters[k] += 1;
      const int f = G.hSc[k].flags;
      if (f & 4) { G.status[k] = PCB_ERR_NONFINITE; G.done[k] = 1; ending[k] = 1; continue; }
      if ((f & 1) || (f & 8) || j + 1 >= c.restart || G.iters[k] >= c.maxit) ending[k] = 1;
      any_end |= ending[k] != 0;
    }
    if (any_end) {   // d = Z y for the instances whose cycle ends at this step (k = j + 1 columns)
      std::vector<int> m2(n, 0);
      for (int k = 0; k < n; ++k) m2[k] = ending[k] && !G.done[k];
      if ((rc = set_active(G, m2))) return rc;
      CK(launch_multiaxpy(G.B, SL_ZBASE, j, SL_XI, -1));
    }
    G.j += 1;
  }
  if (any_end) {
    for (int k = 0; k < n; ++k) if (ending[k]) G.in_round[k] = 0;
    if ((rc = set_active(G, G.in_round))) return rc;
  }
  return PCB_OK;
}

// x += d, r = b - op x, decide per instance
int round_end(BGroup& G, const SolveCfg& c, int max_ref) {
  const int n = (int)G.probs.size();
  std::vector<int> mask(n, 0);
  for (int k = 0; k < n; ++k) mask[k] = G.round_member[k] && !G.done[k];
  int rc;
  if ((rc = set_active(G, mask))) return rc;
  CK(launch_axpby(G.B, AX_ADD, SL_XI, SL_X, -1));
  CK(launch_matvec(G.B, G.op, SL_X, SL_BI, SL_B, EPI_RESID));
  CK(launch_reduce(G.B, G.B.off_mv, 1, 0, SS_NORM, c.tol, 0, 0));
  if ((rc = read_all(G))) return rc;
  for (int k = 0; k < n; ++k) {
    if (!mask[k]) continue;
    G.sweeps[k] += 1;
    G.rnorm[k] = std::sqrt(G.hSc[k].dot1);
    const double rel = G.rnorm[k] / G.bnorm[k];
    if (!std::isfinite(rel)) { G.status[k] = PCB_ERR_NONFINITE; G.done[k] = 1; }
    else if (rel <= c.tol) G.done[k] = 1;
    else if (G.sweeps[k] >= max_ref || G.iters[k] >= c.maxit) { G.status[k] = PCB_NOT_CONVERGED; G.done[k] = 1; }
  }
  G.round_open = false;
  return PCB_OK;
}

}  // namespace

extern "C" int pcb_batch_solve(pcb_problem* const* problems, int count, const pcb_solve_opts* opts,
                               const double* const* b_dev, double* const* x_dev, pcb_solve_info* infos) {
  if (!problems || count < 1 || !b_dev || !x_dev) return PCB_ERR_INVALID_ARG;
  for (int k = 0; k < count; ++k)
    if (!problems[k] || !b_dev[k] || !x_dev[k] || problems[k]->desc.precision != problems[0]->desc.precision ||
        problems[k]->stream != problems[0]->stream)
      return PCB_ERR_INVALID_ARG;
  auto t0 = std::chrono::steady_clock::now();
  // groups by method (and preconditioner)
  std::vector<std::unique_ptr<BGroup>> groups;
  std::vector<SolveCfg> cfgs;
  for (int k = 0; k < count; ++k) {
    SolveCfg c;
    resolve_defaults(problems[k], opts, c);
    if (c.method == PCB_MINRES && c.kind == PCB_PREC_PS) return PCB_ERR_INVALID_ARG;
    if (problems[k]->g.mg_route) return PCB_ERR_UNSUPPORTED;   // multigrid instances solve one at a time
    if (problems[k]->g.fem) return PCB_ERR_UNSUPPORTED;        // finite elements: single problems
    if (problems[k]->g.bc == PCB_BC_NEUMANN && (c.method == PCB_MINRES || c.kind != PCB_PREC_PS))
      return PCB_ERR_UNSUPPORTED;
    BGroup* G = nullptr;
    for (size_t q = 0; q < groups.size(); ++q)
      if (groups[q]->method == c.method && groups[q]->kind == c.kind) G = groups[q].get();
    if (!G) {
      groups.emplace_back(new BGroup());
      G = groups.back().get();
      G->method = c.method; G->kind = c.kind; G->op = c.op; G->prec = c.prec;
      cfgs.push_back(c);
    }
    G->probs.push_back(problems[k]);
    G->idx.push_back(k);
  }
  cudaStream_t st = problems[0]->stream;
  const int max_ref = (opts && opts->max_refinements > 0) ? opts->max_refinements : 10;
  int rc = PCB_OK;
  for (size_t q = 0; q < groups.size() && rc == PCB_OK; ++q) rc = group_setup(*groups[q], cfgs[q], b_dev, x_dev, st);
  for (size_t q = 0; q < groups.size() && rc == PCB_OK; ++q) rc = round_start(*groups[q], cfgs[q]);
  while (rc == PCB_OK) {
    bool work = false;
    for (size_t q = 0; q < groups.size() && rc == PCB_OK; ++q) {
      BGroup& G = *groups[q];
      if (!G.round_open) continue;
      work = true;
      bool any = false;
      for (int v : G.in_round) any |= v != 0;
      if (any) rc = round_step(G, cfgs[q]);
      else {
        rc = round_end(G, cfgs[q], max_ref);
        if (rc == PCB_OK) rc = round_start(G, cfgs[q]);
      }
    }
    if (!work) break;
  }
  if (rc == PCB_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = PCB_ERR_CUDA;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = rc;
  for (auto& Gp : groups) {
    BGroup& G = *Gp;
    for (size_t k = 0; k < G.probs.size(); ++k) {
      const int s2 = rc != PCB_OK ? rc : G.status[k];
      if (infos) {
        pcb_solve_info& I = infos[G.idx[k]];
        std::memset(&I, 0, sizeof(I));
        I.status = s2; I.method = G.method; I.precond = G.kind; I.iterations = G.iters[k];
        I.refinements = G.sweeps[k]; I.relres = G.bnorm[k] > 0 ? G.rnorm[k] / G.bnorm[k] : 0.0; I.seconds = secs;
      }
      if (s2 < 0 && worst >= 0) worst = s2;
      else if (s2 > 0 && worst == PCB_OK) worst = s2;
    }
  }
  return worst;
}

// ---------------------------------------------------------------------------------------------
// Continuous-batching server: fixed slot tables (one per method) whose empty slots contribute no
// blocks to the shared launches; requests join and leave between steps.
// ---------------------------------------------------------------------------------------------
namespace {

enum { PH_FREE = 0, PH_START, PH_ITER, PH_END, PH_DONE };

struct SrvReq {
  pcb_desc desc;
  const double* rhs;
  double* x;
  long long tag;
};

// First-fit sub-allocator over one device reservation: the server reserves its budget once, at
// creation, and carves each admitted request's workspace (one block) out of it, so admitting and
// retiring requests calls neither cudaMalloc nor cudaFree (both of which can stall the device).
// Blocks are 256-byte aligned; adjacent free blocks merge.  Blocks above an eighth of the
// reservation are placed from the top down and the rest from the bottom up, so that the many small
// workspaces do not fragment the room the few large ones need.
class DevArena {
 public:
  ~DevArena() { if (base_) cudaFree(base_); }
  cudaError_t reserve(size_t bytes) {
    bytes &= ~(size_t)255;
    const cudaError_t e = cudaMalloc(&base_, bytes);
    if (e != cudaSuccess) { base_ = nullptr; return e; }
    size_ = bytes;
    free_.clear(); used_.clear();
    free_[0] = bytes;
    return cudaSuccess;
  }
  size_t size() const { return size_; }
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (!base_ || !bytes) return nullptr;
    if (bytes > size_ / 8) {
      for (auto it = free_.rbegin(); it != free_.rend(); ++it) {
        if (it->second < bytes) continue;
        const size_t off = it->first + it->second - bytes;
        if (it->second == bytes) free_.erase(it->first); else it->second -= bytes;
        used_[off] = bytes;
        return base_ + off;
      }
      return nullptr;
    }
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      used_[off] = bytes;
      return base_ + off;
    }
    return nullptr;
  }
  void release(void* ptr) {
    if (!ptr) return;
    const size_t off = (size_t)((char*)ptr - base_);
    auto u = used_.find(off);
    if (u == used_.end()) return;
    size_t o = off, len = u->second;
    used_.erase(u);
    auto next = free_.lower_bound(o);
    if (next != free_.end() && next->first == o + len) { len += next->second; next = free_.erase(next); }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == o) { o = prev->first; len += prev->second; free_.erase(prev); }
    }
    free_[o] = len;
  }

 private:
  char* base_ = nullptr;
  size_t size_ = 0;
  std::map<size_t, size_t> free_;   // offset -> length
  std::map<size_t, size_t> used_;
};

// One request's workspace inside its arena block: tables, preconditioner scratch, the MINRES
// vectors, the refinement pair, the GMRES bases (GMRES requests), and the right-hand side and
// solution; every part 256-byte aligned.
struct SrvLayout {
  size_t tab, scr, minres, mixed, gmres, io, total;
  TableLayout tl;
};

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

void srv_layout(const Geom& g, int method, int restart, SrvLayout& L) {
  const size_t vb = (size_t)2 * g.mn * sizeof(double);
  size_t o = 0;
  L.tab = o; o += up256(table_layout(g, L.tl));
  L.scr = o; o += up256(std::max<size_t>(vb, (size_t)16 * g.n * g.N * (size_t)g.lr));
  L.minres = o; o += 7 * vb;
  L.mixed = o; o += 2 * vb;
  L.gmres = o; o += method == PCB_MINRES ? 0 : (size_t)(2 * restart + 2) * vb;
  L.io = o; o += 2 * vb;
  L.total = up256(o);
}

int srv_method(const pcb_desc& d) { return d.theta == 1.0 && d.bc != PCB_BC_NEUMANN ? PCB_MINRES : PCB_GMRES; }

struct SrvSlot {
  int phase = PH_FREE;
  SrvReq req;
  Geom g;                   // the request's geometry, device pointers into its block
  void* block = nullptr;    // its workspace in the server's arena
  unsigned char* stage = nullptr;   // page-locked staging of its tables (kept with the slot)
  size_t stage_bytes = 0;
  double* b = nullptr;      // device copies of the right-hand side and the solution
  double* x = nullptr;
  double bnorm = 0, rnorm = 0;
  int iters = 0, sweeps = 0, status = PCB_OK;
  bool first = true;
  long long bytes = 0;
};

struct SrvGroup {
  int method = PCB_MINRES, op = PCB_OP_A, kind = PCB_PREC_ABS_PS;
  int cap = 0;
  std::vector<SrvSlot> slots;
  std::vector<Geom> hG;
  std::vector<Slots> hS;
  Geom* dG = nullptr; Slots* dS = nullptr; Scal* dSc = nullptr; int* dAct = nullptr; int* dOff = nullptr;
  double* dPart = nullptr; double* dTol = nullptr;
  Scal* hSc = nullptr; int* hAct = nullptr; double* hTol = nullptr; Slots* hSpin = nullptr;
  Batch B;
  bool dirty = true;
};

}  // namespace

struct pcb_server {
  pcb_server_opts o;
  cudaStream_t st;
  DevArena arena;
  std::vector<SrvReq> queue;   // arrival order; admitted entries are marked taken
  std::vector<char> taken;
  size_t qhead = 0;
  int head_wait = 0;           // steps the oldest queued request has been passed over
  SrvGroup grp[2];             // 0: MINRES (theta = 1), 1: GMRES
  std::vector<pcb_server_done> done;
};

namespace {

long long srv_bytes(const pcb_desc* d, int restart) {
  Geom g;
  init_geom(d, g);
  apply_cached_tuning(g, d->precision);
  SrvLayout L;
  srv_layout(g, srv_method(*d), restart, L);
  return (long long)L.total;
}

int srv_upload(SrvGroup& G, cudaStream_t st) {
  const int n = G.cap;
  if (G.dirty) {
    CK(cudaStreamSynchronize(st));
    std::vector<int> staging;
    int rc = fill_batch(G.B, G.hG, G.dOff, st, staging);
    if (rc) return rc;
    CK(cudaMemcpyAsync(G.dG, G.hG.data(), sizeof(Geom) * n, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    G.B.G = G.dG; G.B.S = G.dS; G.B.Sc = G.dSc; G.B.active = G.dAct; G.B.partial = G.dPart; G.B.tols = G.dTol;
    G.dirty = false;
  }
  CK(cudaStreamSynchronize(st));
  std::memcpy(G.hSpin, G.hS.data(), sizeof(Slots) * n);
  CK(cudaMemcpyAsync(G.dS, G.hSpin, sizeof(Slots) * n, cudaMemcpyHostToDevice, st));
  return PCB_OK;
}

int srv_mask(SrvGroup& G, cudaStream_t st, int phase, bool extra_first = false) {
  CK(cudaStreamSynchronize(st));
  int any = 0;
  for (int k = 0; k < G.cap; ++k) {
    const SrvSlot& s = G.slots[k];
    G.hAct[k] = s.phase == phase && (!extra_first || s.first);
    any |= G.hAct[k];
  }
  CK(cudaMemcpyAsync(G.dAct, G.hAct, sizeof(int) * G.cap, cudaMemcpyHostToDevice, st));
  return any ? 1 : 0;
}

int srv_read(SrvGroup& G, cudaStream_t st) {
  CK(cudaMemcpyAsync(G.hSc, G.dSc, sizeof(Scal) * G.cap, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PCB_OK;
}

int srv_group_step(pcb_server* S, SrvGroup& G) {
  cudaStream_t st = S->st;
  const double tol = S->o.tol;
  const int prec = S->o.precision, restart = S->o.restart;
  int rc;
  bool any = false;
  for (auto& s : G.slots) any |= s.phase != PH_FREE;
  if (!any) return PCB_OK;
  // server requests have a constant coefficient: the transform route of the preconditioner
  auto precond = [&](int in_slot, int out_slot) {
    const cudaError_t e = launch_precond_fast(G.B, G.kind, prec, in_slot, out_slot);
    return e == cudaSuccess ? PCB_OK : cuda_status(e);
  };
  if ((rc = srv_upload(G, st))) return rc;
  // ---- round end: x += d, r = b - op x
  if ((rc = srv_mask(G, st, PH_END)) < 0) return rc;
  if (rc == 1) {
    CK(launch_axpby(G.B, AX_ADD, SL_XI, SL_X, -1));
    CK(launch_matvec(G.B, G.op, SL_X, SL_BI, SL_B, EPI_RESID));
    CK(launch_reduce(G.B, G.B.off_mv, 1, 0, SS_NORM, tol, 0, 0));
    if ((rc = srv_read(G, st))) return rc;
    for (int k = 0; k < G.cap; ++k) {
      SrvSlot& s = G.slots[k];
      if (s.phase != PH_END) continue;
      s.sweeps += 1;
      s.rnorm = std::sqrt(G.hSc[k].dot1);
      const double rel = s.bnorm > 0 ? s.rnorm / s.bnorm : 0.0;
      if (!std::isfinite(rel)) { s.status = PCB_ERR_NONFINITE; s.phase = PH_DONE; }
      else if (rel <= tol) s.phase = PH_DONE;
      else if (s.sweeps >= 10 || s.iters >= S->o.maxit) { s.status = PCB_NOT_CONVERGED; s.phase = PH_DONE; }
      else s.phase = PH_START;
    }
  }
  // ---- round start
  if ((rc = srv_mask(G, st, PH_START, true)) < 0) return rc;
  if (rc == 1) {   // first round: ||b||
    CK(launch_dot(G.B, SL_B, SL_B));
    CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_BNORM, tol, 0, 0));
    if ((rc = srv_read(G, st))) return rc;
    for (int k = 0; k < G.cap; ++k) {
      SrvSlot& s = G.slots[k];
      if (s.phase != PH_START || !s.first) continue;
      s.bnorm = G.hSc[k].bnorm; s.rnorm = s.bnorm; s.first = false;
      if (!std::isfinite(s.bnorm)) { s.status = PCB_ERR_NONFINITE; s.phase = PH_DONE; }
      else if (s.bnorm == 0.0) { s.rnorm = 0.0; s.phase = PH_DONE; }
    }
  }
  if ((rc = srv_mask(G, st, PH_START)) < 0) return rc;
  if (rc == 1) {
    for (int k = 0; k < G.cap; ++k)
      if (G.slots[k].phase == PH_START)
        G.hTol[k] = std::min(0.5, tol * G.slots[k].bnorm / G.slots[k].rnorm);
    CK(cudaMemcpyAsync(G.dTol, G.hTol, sizeof(double) * G.cap, cudaMemcpyHostToDevice, st));
    CK(launch_axpby(G.B, AX_ZERO, -1, SL_XI, -1));
    if (G.method == PCB_MINRES) {
      CK(launch_axpby(G.B, AX_ZERO, -1, SL_W, -1));
      CK(launch_axpby(G.B, AX_ZERO, -1, SL_W2, -1));
      CK(launch_axpby(G.B, AX_COPY, SL_BI, SL_R1, -1));
      CK(launch_axpby(G.B, AX_COPY, SL_BI, SL_R2, -1));
      if ((rc = precond(SL_R2, SL_Y))) return rc;
      CK(launch_dot(G.B, SL_R2, SL_Y));
      CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_MINRES_INIT, tol, 0, 0));
    } else {
      CK(launch_dot(G.B, SL_BI, SL_BI));
      CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_BNORM, tol, 0, 0));
      CK(launch_dot(G.B, SL_BI, SL_BI));
      CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_GMRES_START, tol, 0, 0));
      CK(launch_setslot(G.B, SL_VJ, SL_VBASE, 0, 0));
      CK(launch_axpby(G.B, AX_SCALE_INV_BETA, SL_BI, SL_VJ, -1));
    }
    if ((rc = srv_read(G, st))) return rc;
    for (int k = 0; k < G.cap; ++k) {
      SrvSlot& s = G.slots[k];
      if (s.phase != PH_START) continue;
      const int f = G.hSc[k].flags;
      if (f & 4) { s.status = PCB_ERR_NONFINITE; s.phase = PH_DONE; }
      else if (G.method == PCB_MINRES && (f & 2)) { s.status = PCB_ERR_BREAKDOWN; s.phase = PH_DONE; }
      else s.phase = PH_ITER;
    }
    // device-side slot pointers may have been set by setslot: refresh the host mirror from the rule
    for (int k = 0; k < G.cap; ++k)
      if (G.method != PCB_MINRES && G.slots[k].phase == PH_ITER) G.hS[k].v[SL_VJ] = G.hS[k].v[SL_VBASE];
    if ((rc = srv_upload(G, st))) return rc;
  }
  // ---- one iteration
  if ((rc = srv_mask(G, st, PH_ITER)) < 0) return rc;
  if (rc == 1) {
    std::vector<int> ending(G.cap, 0);
    bool any_end = false;
    if (G.method == PCB_MINRES) {
      CK(launch_matvec(G.B, PCB_OP_A, SL_Y, SL_Q, SL_R1, EPI_MINRES | (prec == PCB_MIXED ? EPI_FAST : 0)));
      CK(launch_reduce(G.B, G.B.off_mv, 1, 0, SS_MINRES_ALFA, tol, 0, 0));
      CK(launch_axpby(G.B, AX_MINRES_R, SL_Q, SL_R2, SL_R1));
      if ((rc = precond(SL_R1, SL_YO))) return rc;
      CK(launch_dot(G.B, SL_R1, SL_YO));
      CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_MINRES_GIVENS, tol, 0, 0));
      CK(launch_minres_wx(G.B, SL_Y, SL_W, SL_W2, SL_XI));
      if ((rc = srv_read(G, st))) return rc;
      for (int k = 0; k < G.cap; ++k) {
        SrvSlot& s = G.slots[k];
        if (s.phase != PH_ITER) continue;
        Slots& H = G.hS[k];
        std::swap(H.v[SL_R1], H.v[SL_R2]); std::swap(H.v[SL_Y], H.v[SL_YO]); std::swap(H.v[SL_W], H.v[SL_W2]);
        s.iters += 1;
        const int f = G.hSc[k].flags;
        if (f & 4) { s.status = PCB_ERR_NONFINITE; s.phase = PH_DONE; }
        else if (f & 2) { s.status = PCB_ERR_BREAKDOWN; s.phase = PH_DONE; }
        else if ((f & 1) || s.iters >= S->o.maxit) s.phase = PH_END;
      }
    } else {
      int jmax = 0;      // largest Arnoldi index among the iterating requests: bounds the basis loops
      for (int k = 0; k < G.cap; ++k) {
        if (G.slots[k].phase != PH_ITER) continue;
        const int j = G.hSc[k].j;
        jmax = std::max(jmax, j);
        const size_t nv = (size_t)2 * G.hG[k].mn;
        Slots& H = G.hS[k];
        H.v[SL_VJ] = H.v[SL_VBASE] + (size_t)j * nv;
        H.v[SL_ZJ] = H.v[SL_ZBASE] + (size_t)j * nv;
        H.v[SL_VJ1] = H.v[SL_VBASE] + (size_t)(j + 1) * nv;
      }
      if ((rc = srv_upload(G, st))) return rc;
      if ((rc = precond(SL_VJ, SL_ZJ))) return rc;
      CK(launch_matvec(G.B, G.op, SL_ZJ, SL_VJ1, -1, EPI_PLAIN));
      for (int pass = 0; pass < 2; ++pass) {
        CK(launch_multidot(G.B, SL_VBASE, -1, SL_VJ1, jmax));
        CK(launch_reduce_multi(G.B, -1, pass));
        CK(launch_multiaxpy(G.B, SL_VBASE, -1, SL_VJ1, pass, jmax));
      }
      CK(launch_dot(G.B, SL_VJ1, SL_VJ1));
      CK(launch_reduce(G.B, G.B.off_vec, 1, 0, SS_GMRES_ARNOLDI, tol, -1, restart));
      CK(launch_axpby(G.B, AX_SCALE_INV_HNORM, SL_VJ1, SL_VJ1, -1));
      if ((rc = srv_read(G, st))) return rc;
      for (int k = 0; k < G.cap; ++k) {
        SrvSlot& s = G.slots[k];
        if (s.phase != PH_ITER) continue;
        s.iters += 1;
        const int f = G.hSc[k].flags;
        if (f & 4) { s.status = PCB_ERR_NONFINITE; s.phase = PH_DONE; continue; }
        if ((f & 1) || (f & 8) || G.hSc[k].j >= restart || s.iters >= S->o.maxit) { ending[k] = 1; any_end = true; }
      }
      if (any_end) {   // d = Z y for the requests whose cycle ends here
        CK(cudaStreamSynchronize(st));
        int jend = 0;    // the update uses columns 0 .. j-1 of each ending request
        for (int k = 0; k < G.cap; ++k) {
          G.hAct[k] = ending[k];
          if (ending[k]) jend = std::max(jend, G.hSc[k].j - 1);
        }
        CK(cudaMemcpyAsync(G.dAct, G.hAct, sizeof(int) * G.cap, cudaMemcpyHostToDevice, st));
        CK(launch_multiaxpy(G.B, SL_ZBASE, -1, SL_XI, -1, jend));
        for (int k = 0; k < G.cap; ++k) if (ending[k]) G.slots[k].phase = PH_END;
      }
    }
  }
  return PCB_OK;
}

}  // namespace

extern "C" {

int pcb_server_create(const pcb_server_opts* o, pcb_server** out) {
  if (!o || !out || o->budget_bytes <= 0 || o->max_slots < 1 || o->max_slots > 256 ||
      (o->precision != PCB_FP64 && o->precision != PCB_MIXED))
    return PCB_ERR_INVALID_ARG;
  pcb_server* S = new (std::nothrow) pcb_server();
  if (!S) return PCB_ERR_OUT_OF_MEMORY;
  S->o = *o;
  if (S->o.tol <= 0) S->o.tol = 1e-8;
  if (S->o.maxit <= 0) S->o.maxit = 500;
  if (S->o.restart <= 0) S->o.restart = 16;
  S->o.restart = std::min(S->o.restart, PCB_MAX_RESTART);
  S->st = (cudaStream_t)o->stream;
  if (upload_constants() != cudaSuccess) { delete S; return PCB_ERR_CUDA; }
  // the budget is reserved here, once (at most what the device has free, less 2 GiB of headroom)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); delete S; return PCB_ERR_CUDA; }
  const size_t head = (size_t)2 << 30;
  const size_t want = std::min<size_t>((size_t)o->budget_bytes, free_b > head ? free_b - head : 0);
  if (want < 256 || S->arena.reserve(want) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return PCB_ERR_OUT_OF_MEMORY;
  }
  for (int q = 0; q < 2; ++q) {
    SrvGroup& G = S->grp[q];
    G.method = q == 0 ? PCB_MINRES : PCB_GMRES;
    G.op = q == 0 ? PCB_OP_A : PCB_OP_AHAT;
    G.kind = q == 0 ? PCB_PREC_ABS_PS : PCB_PREC_PS;
    const int n = G.cap = o->max_slots;
    G.slots.assign(n, SrvSlot());
    Geom empty;
    std::memset(&empty, 0, sizeof(empty));
    G.hG.assign(n, empty);
    Slots es;
    std::memset(&es, 0, sizeof(es));
    G.hS.assign(n, es);
    const size_t part = (size_t)n * 2432 * (PCB_MAX_RESTART + 1) + 1;
    if (cudaMalloc(&G.dG, sizeof(Geom) * n) || cudaMalloc(&G.dS, sizeof(Slots) * n) ||
        cudaMalloc(&G.dSc, sizeof(Scal) * n) || cudaMalloc(&G.dAct, sizeof(int) * n) ||
        cudaMalloc(&G.dOff, sizeof(int) * 10 * (n + 1)) || cudaMalloc(&G.dPart, part * sizeof(double)) ||
        cudaMalloc(&G.dTol, sizeof(double) * n) || cudaMallocHost(&G.hSc, sizeof(Scal) * n) ||
        cudaMallocHost(&G.hAct, sizeof(int) * n) || cudaMallocHost(&G.hTol, sizeof(double) * n) ||
        cudaMallocHost(&G.hSpin, sizeof(Slots) * n)) {
      cudaGetLastError();
      pcb_server_destroy(S);
      return PCB_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(G.dSc, 0, sizeof(Scal) * n);
    std::memset(&G.B, 0, sizeof(Batch));
  }
  *out = S;
  return PCB_OK;
}

void pcb_server_destroy(pcb_server* S) {
  if (!S) return;
  cudaStreamSynchronize(S->st);
  for (int q = 0; q < 2; ++q) {
    SrvGroup& G = S->grp[q];
    for (auto& s : G.slots) if (s.stage) cudaFreeHost(s.stage);
    cudaFree(G.dG); cudaFree(G.dS); cudaFree(G.dSc); cudaFree(G.dAct); cudaFree(G.dOff); cudaFree(G.dPart);
    cudaFree(G.dTol); cudaFreeHost(G.hSc); cudaFreeHost(G.hAct); cudaFreeHost(G.hTol); cudaFreeHost(G.hSpin);
  }
  delete S;   // the arena's reservation is freed with it
}

int pcb_server_submit(pcb_server* S, const pcb_desc* d, const double* rhs, double* x, long long tag) {
  if (!S || !d || !rhs || !x) return PCB_ERR_INVALID_ARG;
  if (d->a_edges || d->fem || d->multigrid) return PCB_ERR_UNSUPPORTED;
  pcb_desc dd = *d;
  dd.precision = S->o.precision;
  dd.stream = (void*)S->st;
  const int rc = validate_desc(&dd);
  if (rc != PCB_OK) return rc;
  const long long need = srv_bytes(&dd, S->o.restart);
  if (need > S->o.budget_bytes || need > (long long)S->arena.size()) return PCB_ERR_TOO_LARGE;
  S->queue.push_back(SrvReq{dd, rhs, x, tag});
  S->taken.push_back(0);
  return PCB_OK;
}

}  // extern "C"

namespace {

// Admit request r into free slot k of group G: carve its workspace from the arena (nullptr
// returned when no block fits), stage and upload its tables, copy its right-hand side.
int srv_admit(pcb_server* S, SrvGroup& G, int k, const SrvReq& r, bool* fitted) {
  *fitted = false;
  Geom g;
  init_geom(&r.desc, g);
  apply_cached_tuning(g, S->o.precision);
  SrvLayout L;
  srv_layout(g, G.method, S->o.restart, L);
  unsigned char* blk = (unsigned char*)S->arena.alloc(L.total);
  if (!blk) return PCB_OK;
  *fitted = true;
  SrvSlot& s = G.slots[k];
  const size_t tab_bytes = L.tl.bytes;
  if (s.stage_bytes < tab_bytes) {
    if (s.stage) cudaFreeHost(s.stage);
    s.stage = nullptr; s.stage_bytes = 0;
    const size_t sz = std::max<size_t>(tab_bytes, 192 * 1024);
    if (cudaMallocHost(&s.stage, sz) != cudaSuccess) { cudaGetLastError(); S->arena.release(blk); return PCB_ERR_OUT_OF_MEMORY; }
    s.stage_bytes = sz;
  }
  fill_tables(&r.desc, g, L.tl, s.stage);
  bind_tables(g, L.tl, blk + L.tab);
  g.scratch = blk + L.scr;
  const size_t nv = (size_t)2 * g.mn;
  s.phase = PH_START; s.req = r; s.g = g; s.block = blk; s.first = true;
  s.b = (double*)(blk + L.io); s.x = s.b + nv;
  s.bnorm = s.rnorm = 0; s.iters = s.sweeps = 0; s.status = PCB_OK;
  s.bytes = (long long)L.total;
  CK(cudaMemcpyAsync(blk + L.tab, s.stage, tab_bytes, cudaMemcpyHostToDevice, S->st));
  CK(copy_host(s.b, r.rhs, nv, true, S->st, nullptr));
  CK(cudaMemsetAsync(s.x, 0, nv * sizeof(double), S->st));
  double* v = (double*)(blk + L.minres);
  double* mixed = (double*)(blk + L.mixed);
  CK(cudaMemcpyAsync(mixed, s.b, nv * sizeof(double), cudaMemcpyDeviceToDevice, S->st));
  Slots& H = G.hS[k];
  std::memset(&H, 0, sizeof(H));
  H.v[SL_R1] = v; H.v[SL_R2] = v + nv; H.v[SL_Y] = v + 2 * nv; H.v[SL_YO] = v + 3 * nv; H.v[SL_Q] = v + 4 * nv;
  H.v[SL_W] = v + 5 * nv; H.v[SL_W2] = v + 6 * nv; H.v[SL_R] = v;
  H.v[SL_BI] = mixed; H.v[SL_XI] = mixed + nv;
  if (G.method != PCB_MINRES) {
    double* gm = (double*)(blk + L.gmres);
    H.v[SL_VBASE] = gm; H.v[SL_ZBASE] = gm + (size_t)(S->o.restart + 1) * nv;
  }
  H.v[SL_X] = s.x; H.v[SL_B] = s.b;
  G.hG[k] = g;
  G.dirty = true;
  return PCB_OK;
}

constexpr int kSrvScan = 256;        // queued requests a step looks at for admission
constexpr int kSrvMaxPass = 64;      // steps the oldest request may be passed over

}  // namespace

extern "C" {

int pcb_server_step(pcb_server* S, pcb_server_done* done, int max_done, int* n_done, int* n_active, int* n_queued) {
  if (!S) return PCB_ERR_INVALID_ARG;
  int rc = PCB_OK;
  // retire: copy the solution to the caller's buffer, return the workspace to the arena
  bool retired = false;
  for (int q = 0; q < 2; ++q) {
    SrvGroup& G = S->grp[q];
    for (int k = 0; k < G.cap; ++k) {
      SrvSlot& s = G.slots[k];
      if (s.phase != PH_DONE) continue;
      if (copy_host(s.req.x, s.x, (size_t)2 * s.g.mn, false, S->st, nullptr) != cudaSuccess) return PCB_ERR_CUDA;
      retired = true;
      pcb_server_done r;
      r.tag = s.req.tag; r.status = s.status; r.iterations = s.iters; r.refinements = s.sweeps;
      r.relres = s.bnorm > 0 ? s.rnorm / s.bnorm : 0.0;
      S->done.push_back(r);
      s.phase = PH_FREE;
      std::memset(&G.hG[k], 0, sizeof(Geom));
      std::memset(&G.hS[k], 0, sizeof(Slots));
      G.dirty = true;
    }
  }
  // the copies above end before any retired block is handed out again or reported done
  if (retired && cudaStreamSynchronize(S->st) != cudaSuccess) return PCB_ERR_CUDA;
  for (int q = 0; q < 2; ++q)
    for (auto& s : S->grp[q].slots)
      if (s.phase == PH_FREE && s.block) { S->arena.release(s.block); s.block = nullptr; }
  // admit: the queued requests in arrival order, each one that finds a free slot of its method and
  // a block in the arena; once the oldest has been passed over kSrvMaxPass steps, only it may enter
  const bool head_only = S->head_wait >= kSrvMaxPass;
  bool head_admitted = false;
  int scanned = 0;
  for (size_t i = S->qhead; i < S->queue.size() && scanned < kSrvScan; ++i) {
    if (S->taken[i]) continue;
    ++scanned;
    const SrvReq& r = S->queue[i];
    SrvGroup& G = S->grp[srv_method(r.desc) == PCB_MINRES ? 0 : 1];
    int free_k = -1;
    for (int k = 0; k < G.cap; ++k) if (G.slots[k].phase == PH_FREE && !G.slots[k].block) { free_k = k; break; }
    bool fitted = false;
    if (free_k >= 0 && (rc = srv_admit(S, G, free_k, r, &fitted)) != PCB_OK) return rc;
    if (fitted) {
      S->taken[i] = 1;
      if (i == S->qhead) head_admitted = true;
    }
    if (head_only) break;
  }
  while (S->qhead < S->queue.size() && S->taken[S->qhead]) { ++S->qhead; head_admitted = true; }
  S->head_wait = (S->qhead < S->queue.size() && !head_admitted) ? S->head_wait + 1 : 0;
  if (S->qhead > 4096 && S->qhead * 2 > S->queue.size()) {
    S->queue.erase(S->queue.begin(), S->queue.begin() + S->qhead);
    S->taken.erase(S->taken.begin(), S->taken.begin() + S->qhead);
    S->qhead = 0;
  }
  // advance every admitted request
  for (int q = 0; q < 2 && rc == PCB_OK; ++q) rc = srv_group_step(S, S->grp[q]);
  if (rc != PCB_OK) return rc;
  int nd = 0;
  while (nd < max_done && !S->done.empty()) {
    done[nd++] = S->done.front();
    S->done.erase(S->done.begin());
  }
  int act = 0;
  for (int q = 0; q < 2; ++q) for (auto& s : S->grp[q].slots) act += s.phase != PH_FREE;
  int queued = 0;
  for (size_t i = S->qhead; i < S->queue.size(); ++i) queued += !S->taken[i];
  if (n_done) *n_done = nd;
  if (n_active) *n_active = act;
  if (n_queued) *n_queued = queued;
  return PCB_OK;
}

}  // extern "C"
