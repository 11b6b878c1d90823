// Measured FP64 instruction rates of this device (pcb_measure_fp64_rates in include/pcb.h): the
// denominators of the rooflines of the FP64-bound steps (the all-at-once product and the Krylov
// vector updates run at the FP64 pipe's rate rather than at the memory's).
//
// Every thread runs kChains independent dependence chains of kIters fused multiply-adds (or adds)
// on register values, so the FP64 pipe, not latency, sets the time; the grid fills the device
// several times over.  The result is written so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include <algorithm>

#include "pcb_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_fp64_fma(double* __restrict__ out, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int k = 0; k < kIters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[blockIdx.x] = s;   // never true for these inputs; keeps the work alive
}

__global__ void __launch_bounds__(256) k_fp64_add(double* __restrict__ out, double b) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int k = 0; k < kIters; ++k) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] + b;
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int pcb_measure_fp64_rates(void* stream, double* fma_per_s, double* add_per_s) {
  if (!fma_per_s || !add_per_s) return PCB_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PCB_ERR_CUDA;
  const int blocks = sms * 16;
  double* out = nullptr;
  if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return PCB_ERR_OUT_OF_MEMORY; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  const double ops = (double)blocks * 256 * kChains * kIters;
  double best[2] = {0.0, 0.0};
  for (int which = 0; which < 2; ++which) {
    for (int rep = 0; rep < 4; ++rep) {        // the first launch warms up; keep the best
      cudaEventRecord(e0, st);
      if (which == 0) k_fp64_fma<<<blocks, 256, 0, st>>>(out, 0.999999, 1e-7);
      else k_fp64_add<<<blocks, 256, 0, st>>>(out, 1e-7);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) { cudaFree(out); return PCB_ERR_CUDA; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0 && ms > 0.f) best[which] = std::max(best[which], ops / (ms * 1e-3));
    }
  }
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  cudaFree(out);
  *fma_per_s = best[0];
  *add_per_s = best[1];
  return cudaGetLastError() == cudaSuccess ? PCB_OK : PCB_ERR_CUDA;
}
