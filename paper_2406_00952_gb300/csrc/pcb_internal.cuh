// Internal definitions shared by the CUDA translation units of libpcb.
//
// Every kernel is written for a *batch* of independent problem instances: a launch covers
// the blocks of all instances, `blk_off[k]..blk_off[k+1]` being instance k's blocks.  A single
// problem is a batch of one.  Per-instance constants live in `Geom`, per-instance vector
// pointers in `Slots` (device memory, so a solver can rotate them on the device), per-instance
// Krylov scalars in `Scal`.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/pcb.h"

#define PCB_MAX_STAGES 12
#define PCB_NSLOTS 24
#define PCB_MAX_RESTART 32

namespace pcb {

// ------------------------------------------------------------------------------------------
// per-device host state.  Kernel attributes (the dynamic shared-memory limit), __constant__
// tables and occupancy figures belong to a device, so each device the library runs on needs its
// own setup: a process-wide "done" flag would leave a second device unconfigured.
// ------------------------------------------------------------------------------------------
constexpr int kMaxDevices = 64;

// Runs f() the first time the current device reaches this flag (again after a failure).  Two
// host threads may both run f() for the same device at first, so f() must be idempotent.
struct DeviceOnce {
  std::atomic<unsigned long long> mask{0};
  template <typename F>
  cudaError_t operator()(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < kMaxDevices) ? 1ull << dev : 0ull;
    if (bit && (mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = f();
    if (e == cudaSuccess && bit) mask.fetch_or(bit, std::memory_order_acq_rel);
    return e;
  }
};

// A per-device integer computed once (0 = not yet known).
struct DeviceInt {
  std::atomic<int> v[kMaxDevices] = {};
  template <typename F>
  cudaError_t get(int* out, F&& compute) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return compute(out);
    int x = v[dev].load(std::memory_order_acquire);
    if (!x) {
      if ((e = compute(&x)) != cudaSuccess) return e;
      v[dev].store(x, std::memory_order_release);
    }
    *out = x;
    return cudaSuccess;
  }
};

// the dynamic shared-memory limit of kernel `k`, once per device
template <typename K>
cudaError_t set_smem_limit(DeviceOnce& once, K k, int bytes) {
  return once([&] { return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes); });
}

// ------------------------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ------------------------------------------------------------------------------------------
template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };
template <typename R> using cx = typename Cx<R>::T;

template <typename R> __host__ __device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> c; c.x = a; c.y = b; return c; }
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { T c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { T c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename T> __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
template <typename T, typename R> __device__ __forceinline__ T cscale(T a, R s) { a.x *= s; a.y *= s; return a; }
// FP32 pairs: one packed instruction (f32x2, sm_100 and later) per complex add, subtract or real
// scale; each lane rounds exactly like the scalar operation (a - b = fma(-1, b, a) is exact
// before its single rounding)
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
// s * v + a for a real s
template <typename T, typename R> __device__ __forceinline__ T cfma_s(R s, T v, T a) {
  a.x = fma(s, v.x, a.x); a.y = fma(s, v.y, a.y); return a;
}
__device__ __forceinline__ float2 cfma_s(float s, float2 v, float2 a) { return __ffma2_rn(make_float2(s, s), v, a); }
// a * (-i)
template <typename T> __device__ __forceinline__ T cmul_mi(T a) { T c; c.x = a.y; c.y = -a.x; return c; }
// a * (+i)
template <typename T> __device__ __forceinline__ T cmul_pi(T a) { T c; c.x = -a.y; c.y = a.x; return c; }

// ------------------------------------------------------------------------------------------
// per-instance geometry and tables
// ------------------------------------------------------------------------------------------
struct FftPlan {
  int M;                          // transform length
  int nst;                        // number of Stockham stages
  int rad[PCB_MAX_STAGES];        // radix of each stage (2, 3, 4 or 8)
};

struct Geom {
  int N, n, m;                    // m = N*N
  int L, M;                       // L = N+1 (DST-I order; Neumann: N-1, DCT-I order), M = 2L (extended FFT length)
  int bc;                         // PCB_BC_DIRICHLET or PCB_BC_NEUMANN (mirrored stencil, DCT-I transform)
  long long mn;                   // m*n (one half of the all-at-once vector)
  double theta, tau, gamma, alpha, h, sqrt_gamma;
  double zeta;                    // omega = exp(i zeta)
  int zeta_pi;                    // 1 when zeta = pi: the two halves share one complex time line
  double c;                       // tau a / h^2 (a: the constant coefficient)
  int var_a;                      // 0: a = 1; 1: coefficient tables below
  int mg_route;                   // 1: the shifted solves of the preconditioners run as multigrid V-cycles
                                  //    (variable a, or on request with a constant one)
  int fem;                        // 1: Q1 finite elements (spatial operator M^{-1/2} K M^{-1/2}, applied
                                  //    through the DST-I; kap holds its 1D eigenvalues a kappa1_p / mu_p)
  // FP32 scratch layout of the pipelined passes: rows of lr values (lr = L + 16 when the pipelined
  // DST runs: 64-byte aligned rows, stride off a power of two; else N), slices of mp = N lr values;
  // buffer b, half h, time t, row r, index i at (float*)scratch + (2b + h) n mp + t mp + r lr + i
  int lr;
  long long mp;
  // launch shapes (blocks of each pass for this instance)
  // launch shapes of the preconditioner passes, index 0 = FP64 apply, 1 = FP32 apply
  int dst_lpb[2];                 // lines per block of the x1-line DST pass
  int dst_lpb_j[2];               // lines per block of the x2-line DST pass
  int dst_q, time_q;              // values per lane of the register FFTs (line length / lanes)
  int dst_blocks_i[2], dst_blocks_j[2]; // blocks of the x1-line and x2-line DST passes
  int time_cpb[2];                // spatial columns per block of the time pass
  int time_blocks[2];
  int tune;                       // kernel choices of the autotuner (TUNE_* bits; 0 = defaults)
  int mv_tchunk;                  // time steps per thread in the theta = 1 matvec
  int mv_blocks;                  // blocks of the matvec
  int vec_blocks;                 // blocks of the vector kernels over 2mn
  FftPlan pdst, ptime;
  // tables (device)
  const double* kap;              // N: eigenvalues a kappa_p of the 1D second difference (Dirichlet p = 1..N,
                                  //    Neumann k = 0..N-1); finite elements: of M1^{-1/2} K1 M1^{-1/2}
  const double* mass;             // fem: N eigenvalues mu_p of the 1D mass matrix (h/6) tridiag(1, 4, 1)
  const double2* mu_d;            // n: lambda(S_n) at F-slot r (FP64)
  const float2* mu_f;
  const double2* twd_d;           // M: exp(-2 pi i k / M)
  const float2* twd_f;
  const double2* twt_d;           // n: exp(-2 pi i k / n)
  const float2* twt_f;
  const double2* pre_d;           // n: exp(-i pi t / n)   (zeta = pi scaling, D_omega conj)
  const float2* pre_f;
  const double* axs;              // var_a: tau/h^2 * ax  (N x (N+1))
  const double* ays;              //        tau/h^2 * ay  ((N+1) x N)
  const double* dgs;              //        tau/h^2 * (sum of the 4 edge coefficients) (N x N)
  void* scratch;                  // preconditioner workspace: 2mn values of the apply's Real type
  const void* mg;                 // multigrid workspace (variable a), else null
};

// Autotuner choices (Geom::tune): kernel families the FP32 apply may not use, and the tile-size
// scale of the tile kernels (bits 4-5: 0 = default, 1 = half, 2 = double the per-tile element budget)
enum { TUNE_NO_PIPE_DST = 1, TUNE_NO_PIPE_TIME = 2, TUNE_NO_HANDOFF = 4, TUNE_TIME512_3BLK = 8,
       TUNE_TIME512_4BLK = 64 };
__host__ __device__ inline int tune_budget_shift(int tune) { return (tune >> 4) & 3; }

// per-instance Krylov scalars (MINRES and GMRES share the struct)
struct Scal {
  // MINRES (Paige-Saunders recurrences)
  double beta, oldb, alfa, dbar, epsln, oldeps, phibar, cs, sn, delta, gbar, gamma, phi;
  double beta1, bnorm, est;
  // reductions land here
  double dot0, dot1;
  // GMRES
  double H[(PCB_MAX_RESTART + 1) * 2];   // current Hessenberg column (two passes of CGS2)
  double hcol[PCB_MAX_RESTART + 1];
  double R[(PCB_MAX_RESTART + 1) * PCB_MAX_RESTART];   // rotated Hessenberg (column major)
  double g[PCB_MAX_RESTART + 1];
  double gcs[PCB_MAX_RESTART], gsn[PCB_MAX_RESTART];
  double y[PCB_MAX_RESTART];
  double hnorm;
  int itn;          // iterations done
  int j;            // Arnoldi index within the restart cycle
  int active;       // 1 while the instance still iterates
  int flags;        // bit 0: estimate below tolerance; bit 1: breakdown; bit 2: nonfinite
};

struct Slots { double* v[PCB_NSLOTS]; };

// ------------------------------------------------------------------------------------------
// batch -> instance lookup
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int find_inst(const int* __restrict__ off, int count, int b) {
  int lo = 0, hi = count;            // off[lo] <= b < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= b) lo = mid; else hi = mid;
  }
  return lo;
}

// Instance selection of a preconditioner launch: instances with active[k] == 0 are skipped, and
// when fam is set, so are instances whose kernel family fam[k] differs from want.
struct Sel {
  const int* active;
  const int* fam;
  int want;
  __device__ __forceinline__ bool skip(int k) const {
    return (active && !__ldg(active + k)) || (fam && __ldg(fam + k) != want);
  }
};

// family code <-> bit of Batch::fam_*_set: 0 -> 0, P -> log2 P, + 6 with flag 64 (time-major
// hand-off), + 12 with flag 128 (DCT-I lines), + 24 with flag 256 (general-zeta time pass, never
// with 64 or 128); at most kFamilies bits
constexpr int kFamilies = 30;
// (general zeta, flag 256, has P <= 16: indices 24 + log2 P, and 29 for P = 16 with the
// time-major hand-off, the only P it serves)
__host__ __device__ inline int fam_index(int code) {
  if (!code) return 0;
  int b = 0;
  while ((2 << b) <= (code & 63)) ++b;
  if (code & 256) return (code & 64) ? 29 : 24 + b;
  return b + ((code & 64) ? 6 : 0) + ((code & 128) ? 12 : 0);
}
__host__ __device__ inline int fam_code(int index) {
  if (index == 0) return 0;
  if (index == 29) return 16 | 64 | 256;
  if (index >= 24) return (1 << (index - 24)) | 256;
  const int ev = index >= 12 ? 128 : 0;
  if (ev) index -= 12;
  const int tm = index >= 6 ? 64 : 0;
  if (tm) index -= 6;
  return (1 << index) | tm | ev;
}

// ------------------------------------------------------------------------------------------
// host-side launch helpers (defined in runtime.cu)
// ------------------------------------------------------------------------------------------
struct Batch {
  int count;
  const Geom* G;          // device array [count]
  Slots* S;               // device array [count]
  Scal* Sc;               // device array [count]
  const int* active;      // device array [count] or null: 0 => skip instance
  cudaStream_t stream;
  // block offsets for each pass kind (device arrays [count+1]) and totals
  const int* off_dst_i[2]; int tot_dst_i[2];
  const int* off_dst_j[2]; int tot_dst_j[2];
  const int* off_time[2];  int tot_time[2];
  const int* off_mv;    int tot_mv;
  const int* off_vec;   int tot_vec;
  double* partial;        // reduction partials
  const double* tols;     // per-instance tolerances for the scalar steps (device) or null
  int dst_q, time_q;      // register-FFT variant shared by every instance of the batch
  // FP32 kernel families: pipe_pd / pipe_pt > 0 is the family code of the pipelined DST / time
  // kernels (precond_pipe.cu) shared by every instance with work: the lanes per line P, plus 64
  // when pass 2 hands the time pass contiguous time lines (n = 512), plus 128 for DCT-I lines.  0 means the kernels of
  // precond.cu for all, -1 a mix: one launch per family present, each selecting its instances by
  // fam_dst / fam_time (device arrays [count] of codes).  fam_*_set: bit fam_index(code).
  int pipe_pd, pipe_pt;
  const int* fam_dst;
  const int* fam_time;
  int fam_dst_set, fam_time_set;
  int t512v;              // 1 / 2: the n = 512 time pass runs its three / four-blocks-per-SM variant
                          // (every instance of the batch that takes that pass chose it)
  int fem_m;              // > 0: a single finite-element instance with m = fem_m spatial points
                          // (products through the DST-I)
  const int* filt;        // family filter of the launch being issued (null: none)
  int filt_want;
  Sel sel() const { Sel s; s.active = active; s.fam = filt; s.want = filt_want; return s; }
  size_t dst_smem[2], time_smem[2];   // dynamic shared memory per block, per precision
};

}  // namespace pcb
