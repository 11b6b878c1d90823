// Allocation-free preconditioner apply (pcb_precond_apply_noalloc in include/pcb.h).
//
// Some callers cannot call cudaMalloc: code running where the device allocator is off limits
// (an allocator hook, a memory-capped or pre-partitioned process, a real-time loop that must not
// touch the allocator), or plain C callers that want no handle to own and free.  This entry point
// takes a descriptor and the caller's input/output buffers and needs nothing else: its problem
// description, spectral tables and transform scratch live in one file-scope device array of
// PCB_NOALLOC_ARENA_BYTES, which every GPU that loads the library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in for the symbol; its device address
// comes from cudaGetSymbolAddress, once per device, with that device current.  The first call on
// a device performs that look-up and uploads the transforms' constant tables.  Every call copies
// its small descriptor and spectral tables from host memory with cudaMemcpyAsync (pageable
// source), so the host may wait for earlier work on the stream, and no call may be made while
// the stream is being captured into a graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "pcb_internal.cuh"

namespace pcb {
struct TableLayout { size_t kap, mud, muf, twdd, twdf, twtd, twtf, pred, pref, ax, ay, dg, ms, bytes; };
int validate_desc(const pcb_desc* d);
void init_geom(const pcb_desc* d, Geom& g);
size_t table_layout(const Geom& g, TableLayout& t);
void fill_tables(const pcb_desc* d, const Geom& g, const TableLayout& t, unsigned char* host);
void bind_tables(Geom& g, const TableLayout& t, unsigned char* tb);
cudaError_t upload_constants();
size_t dst_smem_bytes(const Geom& g, int p);
size_t time_smem_bytes(const Geom& g, int p);
cudaError_t launch_precond_fast(const Batch& B, int kind, int prec, int in_slot, int out_slot);
}  // namespace pcb

using namespace pcb;

namespace {

// The arena: [Geom | Slots | block offsets | tables | transform scratch], 256-byte aligned parts.
static __device__ __align__(256) unsigned char g_arena[PCB_NOALLOC_ARENA_BYTES];

std::mutex g_mu;                                  // serialises the host side of calls
unsigned char* g_arena_dev[kMaxDevices] = {};     // device address of g_arena, per device
constexpr size_t kTableHostBytes = 160 * 1024;    // largest table set (N = 511, n = 1024) fits
unsigned char g_table_host[kTableHostBytes];

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

int arena_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PCB_ERR_CUDA;
  if (!g_arena_dev[dev]) {
    // once per device: the arena's device address and the transforms' __constant__ tables
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_arena) != cudaSuccess || !ptr) { cudaGetLastError(); return PCB_ERR_CUDA; }
    if (upload_constants() != cudaSuccess) { cudaGetLastError(); return PCB_ERR_CUDA; }
    g_arena_dev[dev] = (unsigned char*)ptr;
  }
  *out = g_arena_dev[dev];
  return PCB_OK;
}

}  // namespace

extern "C" int pcb_precond_apply_noalloc(const pcb_desc* desc, int kind, int precision, const double* x_dev,
                                         double* y_dev) {
  if (!desc || !x_dev || !y_dev) return PCB_ERR_INVALID_ARG;
  if (kind != PCB_PREC_ABS_PS && kind != PCB_PREC_PS && kind != PCB_PREC_PMS) return PCB_ERR_INVALID_ARG;
  if (precision != PCB_FP64 && precision != PCB_MIXED) return PCB_ERR_INVALID_ARG;
  int rc = validate_desc(desc);
  if (rc != PCB_OK) return rc;
  if (desc->a_edges) return PCB_ERR_UNSUPPORTED;     // the multigrid route needs its own workspace
  if (desc->fem) return PCB_ERR_UNSUPPORTED;         // finite elements: the allocating entry points only
  if (desc->bc == PCB_BC_NEUMANN && kind != PCB_PREC_PS) return PCB_ERR_UNSUPPORTED;   // GMRES route only

  Geom g;
  init_geom(desc, g);
  // the arena holds one FP32 scratch buffer of 2mn values: unpadded layout, kernels of precond.cu
  g.lr = g.N;
  g.mp = g.m;
  g.time_blocks[1] = (g.m + g.time_cpb[1] - 1) / g.time_cpb[1];
  TableLayout lay;
  const size_t tab = table_layout(g, lay);
  const size_t real = precision == PCB_MIXED ? sizeof(float) : sizeof(double);
  const size_t o_geom = 0, o_slots = up256(sizeof(Geom)), o_off = o_slots + up256(sizeof(Slots));
  const size_t o_tab = o_off + up256(16 * sizeof(int)), o_scr = o_tab + up256(tab);
  const size_t need = o_scr + up256((size_t)2 * g.mn * real);
  if (need > (size_t)PCB_NOALLOC_ARENA_BYTES || tab > kTableHostBytes) return PCB_ERR_TOO_LARGE;

  std::lock_guard<std::mutex> lock(g_mu);
  unsigned char* base = nullptr;
  if ((rc = arena_for_current_device(&base)) != PCB_OK) return rc;
  cudaStream_t st = (cudaStream_t)desc->stream;

  fill_tables(desc, g, lay, g_table_host);
  bind_tables(g, lay, base + o_tab);
  g.scratch = base + o_scr;      // fully overwritten by every apply: nothing needs clearing
  Slots s;
  std::memset(&s, 0, sizeof(s));
  s.v[0] = (double*)x_dev;
  s.v[1] = y_dev;
  // one instance: each pass's block offsets are {0, blocks}
  int offs[16] = {0, g.dst_blocks_i[0], 0, g.dst_blocks_i[1], 0, g.dst_blocks_j[0], 0, g.dst_blocks_j[1],
                  0, g.time_blocks[0], 0, g.time_blocks[1], 0, g.mv_blocks, 0, g.vec_blocks};
  if (cudaMemcpyAsync(base + o_geom, &g, sizeof(Geom), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + o_slots, &s, sizeof(Slots), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + o_off, offs, sizeof(offs), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + o_tab, g_table_host, tab, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return PCB_ERR_CUDA;
  Batch B;
  std::memset(&B, 0, sizeof(B));
  const int* doff = (const int*)(base + o_off);
  B.count = 1;
  B.G = (const Geom*)(base + o_geom);
  B.S = (Slots*)(base + o_slots);
  B.stream = st;
  for (int p = 0; p < 2; ++p) {
    B.off_dst_i[p] = doff + 0 + 2 * p;  B.tot_dst_i[p] = g.dst_blocks_i[p];
    B.off_dst_j[p] = doff + 4 + 2 * p;  B.tot_dst_j[p] = g.dst_blocks_j[p];
    B.off_time[p] = doff + 8 + 2 * p;   B.tot_time[p] = g.time_blocks[p];
    B.dst_smem[p] = dst_smem_bytes(g, p);
    B.time_smem[p] = time_smem_bytes(g, p);
  }
  B.dst_q = g.dst_q;
  B.time_q = g.time_q;
  B.pipe_pd = 0;
  B.pipe_pt = 0;
  // (copies from pageable host memory return once the source has been staged, so the host buffers
  // above may be reused as soon as cudaMemcpyAsync returns)
  const cudaError_t e = launch_precond_fast(B, kind, precision, 0, 1);
  return e == cudaSuccess ? PCB_OK : PCB_ERR_CUDA;
}
