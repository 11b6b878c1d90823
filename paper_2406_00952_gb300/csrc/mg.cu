// Multigrid preconditioner route for variable a(x) (Sec. 3.5, Step 2 with multigrid).
#include "pcb_internal.cuh"

namespace pcb {

bool mg_available() { return false; }
int mg_launch_count(int kind) { (void)kind; return 0; }
size_t mg_workspace_bytes(const Geom& g) { (void)g; return 256; }
cudaError_t mg_setup(Geom& g, void* ws, const double* a_edges_host) {
  (void)g; (void)ws; (void)a_edges_host;
  return cudaSuccess;
}
cudaError_t launch_precond_mg(const Batch& B, int kind, int prec, int in_slot, int out_slot) {
  (void)B; (void)kind; (void)prec; (void)in_slot; (void)out_slot;
  return cudaErrorNotSupported;
}

}  // namespace pcb
