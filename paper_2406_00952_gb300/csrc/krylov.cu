// Krylov vector kernels and per-instance scalar recurrences, all on the device so an iteration
// needs no host round trip.  Sec. 4 of the paper uses MINRES (symmetric A, SPD preconditioner)
// and GMRES; the scalar recurrences are the textbook ones:
//   MINRES  (Paige & Saunders 1975): preconditioned Lanczos, Givens QR, three-term directions;
//   FGMRES  (Saad 1993): right preconditioning with the preconditioned basis stored, Arnoldi by
//           classical Gram-Schmidt applied twice, Givens rotations on the Hessenberg column.
// Reductions are deterministic: each block of an instance writes one partial for a fixed slice
// of the vector, and one block per instance adds the partials in a fixed order, so a result does
// not depend on which other instances share the launch.
#include <math.h>

#include "pcb_internal.cuh"

namespace pcb {

enum { SS_NONE = 0, SS_MINRES_INIT, SS_MINRES_ALFA, SS_MINRES_GIVENS, SS_NORM, SS_GMRES_ARNOLDI, SS_GMRES_START,
       SS_BNORM };

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;   // valid in thread 0
}

#define INST_PROLOGUE                                              \
  const int inst = find_inst(off, count, blockIdx.x);             \
  if (active && !active[inst]) return;                            \
  const Geom& g = G[inst];                                         \
  const int lb = blockIdx.x - off[inst];                           \
  const long long len = 2 * g.mn;                                  \
  const long long stride = (long long)g.vec_blocks * blockDim.x;   \
  const long long e0 = (long long)lb * blockDim.x + threadIdx.x;

// partial[blk] = sum a.b over the instance's slice
__global__ void __launch_bounds__(256) k_dot(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                             const int* __restrict__ off, int count, const int* __restrict__ active,
                                             int sa, int sb, double* __restrict__ partial) {
  INST_PROLOGUE
  const double* __restrict__ a = S[inst].v[sa];
  const double* __restrict__ b = S[inst].v[sb];
  double acc = 0.0;
  for (long long e = e0; e < len; e += stride) acc = fma(a[e], b[e], acc);
  const double r = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// y = a*x + b*y with (a, b) chosen by `mode` from the instance scalars
enum { AX_COPY = 0, AX_MINRES_R = 1, AX_SCALE_INV_BETA = 2, AX_SCALE_INV_HNORM = 3, AX_ADD = 4, AX_ZERO = 5 };
__global__ void __launch_bounds__(256) k_axpby(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                               const Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                               const int* __restrict__ active, int mode, int sx, int sy, int sz) {
  INST_PROLOGUE
  const Scal& c = Sc[inst];
  const double* __restrict__ x = sx >= 0 ? S[inst].v[sx] : nullptr;
  double* __restrict__ y = S[inst].v[sy];
  if (mode == AX_COPY) {
    for (long long e = e0; e < len; e += stride) y[e] = x[e];
  } else if (mode == AX_MINRES_R) {
    // z = x - (alfa/beta) y  written to slot sz  (x = q, y = r2, z = r1 slot)
    double* __restrict__ z = S[inst].v[sz];
    const double f = -c.alfa / c.beta;
    for (long long e = e0; e < len; e += stride) z[e] = fma(f, y[e], x[e]);
  } else if (mode == AX_SCALE_INV_BETA) {
    const double f = 1.0 / c.beta;
    for (long long e = e0; e < len; e += stride) y[e] = x[e] * f;
  } else if (mode == AX_SCALE_INV_HNORM) {
    const double f = 1.0 / c.hnorm;
    for (long long e = e0; e < len; e += stride) y[e] = x[e] * f;
  } else if (mode == AX_ADD) {
    for (long long e = e0; e < len; e += stride) y[e] += x[e];
  } else {   // AX_ZERO
    for (long long e = e0; e < len; e += stride) y[e] = 0.0;
  }
}

// MINRES direction and solution update:
//   w_new = (y/oldb - oldeps*w2 - delta*w)/gamma  -> slot w2 ;  x += phi*w_new
__global__ void __launch_bounds__(256) k_minres_wx(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                   const Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                   const int* __restrict__ active, int sy, int sw, int sw2, int sx) {
  INST_PROLOGUE
  const Scal& c = Sc[inst];
  const double* __restrict__ y = S[inst].v[sy];
  const double* __restrict__ w = S[inst].v[sw];
  double* __restrict__ w2 = S[inst].v[sw2];
  double* __restrict__ x = S[inst].v[sx];
  // the 1/gamma scale is folded into the three coefficients: four FP64 operations per value (the
  // kernel sits at the FP64 instruction limit as much as at the HBM limit)
  const double ig = 1.0 / c.gamma;
  const double cy = ig / c.oldb, c2 = -c.oldeps * ig, c1 = -c.delta * ig, phi = c.phi;
  for (long long e = e0; e < len; e += stride) {
    double t = y[e] * cy;
    t = fma(c2, w2[e], t);
    t = fma(c1, w[e], t);
    w2[e] = t;
    x[e] = fma(phi, t, x[e]);
  }
}

// CGS: partial[blk*(PCB_MAX_RESTART+1) + i] = V_i . W,  i = 0..j.  JB >= j + 1 bounds the unrolled
// basis loop: the host picks the smallest of 2, 4, 8, 16, 33 that covers the Arnoldi index, so an
// early step does not pay for 33 predicated basis vectors per element.
template <int JB>
__global__ void __launch_bounds__(256) k_multidot(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                  const Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                  const int* __restrict__ active, int svbase, int j, int sw,
                                                  double* __restrict__ partial) {
  INST_PROLOGUE
  if (j < 0) j = Sc[inst].j;   // each instance at its own Arnoldi index
  const double* __restrict__ V = S[inst].v[svbase];
  const double* __restrict__ W = S[inst].v[sw];
  double acc[JB];
#pragma unroll
  for (int i = 0; i < JB; ++i) acc[i] = 0.0;
  for (long long e = e0; e < len; e += stride) {
    const double w = W[e];
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) acc[i] = fma(V[(long long)i * len + e], w, acc[i]);
  }
#pragma unroll
  for (int i = 0; i < JB; ++i) {
    if (i > j) break;
    const double r = block_sum(acc[i]);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * (PCB_MAX_RESTART + 1) + i] = r;
  }
}

// W -= sum_i h_i V_i (coef from Scal.H[pass*(MAX+1) + i]) ; or X += sum_i y_i Z_i (pass = -1)
template <int JB>
__global__ void __launch_bounds__(256) k_multiaxpy(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                   const Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                   const int* __restrict__ active, int svbase, int j, int sw,
                                                   int pass) {
  INST_PROLOGUE
  const Scal& c = Sc[inst];
  if (j < 0) j = pass >= 0 ? c.j : c.j - 1;   // per-instance index (after Arnoldi, c.j = columns)
  const double* __restrict__ V = S[inst].v[svbase];
  double* __restrict__ W = S[inst].v[sw];
  double coef[JB];
#pragma unroll
  for (int i = 0; i < JB; ++i) {
    double h = 0.0;
    if (i <= j) h = pass >= 0 ? -c.H[pass * (PCB_MAX_RESTART + 1) + i] : c.y[i];
    coef[i] = h;
  }
  for (long long e = e0; e < len; e += stride) {
    double w = W[e];
#pragma unroll
    for (int i = 0; i < JB; ++i)
      if (i <= j) w = fma(coef[i], V[(long long)i * len + e], w);
    W[e] = w;
  }
}

// ------------------------------------------------------------------------------------------
// per-instance reductions + scalar steps (one block per instance)
// ------------------------------------------------------------------------------------------
__device__ void scalar_step(Scal& c, int step, double v, double tol, int j, int restart) {
  switch (step) {
    case SS_BNORM:
      c.bnorm = sqrt(v);
      break;
    case SS_NORM:           // true-residual norm: must not touch the Lanczos scalars
      c.dot1 = v;
      break;
    case SS_MINRES_INIT: {
      c.itn = 0; c.flags = 0; c.active = 1;
      if (!isfinite(v)) { c.flags |= 4; c.active = 0; break; }
      if (v < 0.0) { c.flags |= 2; c.active = 0; break; }
      if (v == 0.0) { c.beta1 = 0.0; c.beta = 0.0; c.est = 0.0; c.flags |= 1; c.active = 0; break; }
      c.beta1 = sqrt(v); c.beta = c.beta1; c.oldb = 0.0; c.dbar = 0.0; c.epsln = 0.0; c.phibar = c.beta1;
      c.cs = -1.0; c.sn = 0.0; c.est = 1.0;
      break;
    }
    case SS_MINRES_ALFA:
      c.alfa = v;
      break;
    case SS_MINRES_GIVENS: {
      c.oldb = c.beta;
      if (!(v >= 0.0)) { c.flags |= isfinite(v) ? 2 : 4; c.active = 0; break; }
      c.beta = sqrt(v);
      c.oldeps = c.epsln;
      c.delta = c.cs * c.dbar + c.sn * c.alfa;
      c.gbar = c.sn * c.dbar - c.cs * c.alfa;
      c.epsln = c.sn * c.beta;
      c.dbar = -c.cs * c.beta;
      c.gamma = hypot(c.gbar, c.beta);
      if (c.gamma == 0.0) { c.flags |= 2; c.active = 0; break; }
      c.cs = c.gbar / c.gamma;
      c.sn = c.beta / c.gamma;
      c.phi = c.cs * c.phibar;
      c.phibar = c.sn * c.phibar;
      c.itn += 1;
      c.est = c.phibar / c.beta1;
      if (c.est <= tol) c.flags |= 1;
      if (!isfinite(c.est)) { c.flags |= 4; c.active = 0; }
      break;
    }
    case SS_GMRES_START: {
      // v = ||r||^2 ; beta = ||r|| ; g = (beta, 0, ...); a new cycle clears the previous flags
      c.flags = 0;
      c.itn = 0;
      c.beta = sqrt(v);
      for (int i = 0; i <= PCB_MAX_RESTART; ++i) c.g[i] = 0.0;
      c.g[0] = c.beta;
      c.j = 0;
      c.est = c.beta / c.bnorm;
      if (!isfinite(v)) { c.flags |= 4; c.active = 0; }
      break;
    }
    case SS_GMRES_ARNOLDI: {
      // v = ||w||^2 after two CGS passes; column j of H = H[0][.] + H[1][.]
      const int M1 = PCB_MAX_RESTART + 1;
      double* col = c.R + (long long)j * M1;
      for (int i = 0; i <= j; ++i) col[i] = c.H[i] + c.H[M1 + i];
      const double hn = sqrt(v);
      col[j + 1] = hn;
      c.hnorm = hn;
      for (int i = 0; i < j; ++i) {
        const double t = c.gcs[i] * col[i] + c.gsn[i] * col[i + 1];
        col[i + 1] = -c.gsn[i] * col[i] + c.gcs[i] * col[i + 1];
        col[i] = t;
      }
      double cs = 1.0, sn = 0.0;
      if (col[j + 1] != 0.0) {
        const double r = hypot(col[j], col[j + 1]);
        cs = col[j] / r; sn = col[j + 1] / r;
      }
      c.gcs[j] = cs; c.gsn[j] = sn;
      col[j] = cs * col[j] + sn * col[j + 1];
      col[j + 1] = 0.0;
      c.g[j + 1] = -sn * c.g[j];
      c.g[j] = cs * c.g[j];
      c.itn += 1;
      c.j = j + 1;
      c.est = fabs(c.g[j + 1]) / c.bnorm;
      if (c.est <= tol) c.flags |= 1;
      if (hn == 0.0) c.flags |= 8;        // lucky breakdown: the cycle ends here
      if (!isfinite(c.est)) { c.flags |= 4; c.active = 0; }
      // back substitution for the cycle's coefficients (used when the cycle ends)
      const int k = j + 1;
      for (int i = k - 1; i >= 0; --i) {
        double s = c.g[i];
        for (int q = i + 1; q < k; ++q) s -= c.R[(long long)q * M1 + i] * c.y[q];
        c.y[i] = s / c.R[(long long)i * M1 + i];
      }
      break;
    }
    default:
      break;
  }
  (void)restart;
}

// Sum the instance's partials (nper values per block, index `which`) and run a scalar step.
__global__ void __launch_bounds__(256) k_reduce(const int* __restrict__ off, int count, const int* __restrict__ active,
                                                const double* __restrict__ partial, int nper, int which, Scal* Sc,
                                                int step, double tol, const double* __restrict__ tols, int j,
                                                int restart) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  if (active && !active[inst]) return;
  const int b0 = off[inst], b1 = off[inst + 1];
  double acc = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) acc += partial[(long long)b * nper + which];
  const double s = block_sum(acc);
  if (threadIdx.x == 0) scalar_step(Sc[inst], step, s, tols ? tols[inst] : tol, j < 0 ? Sc[inst].j : j, restart);
}

// multi-reduction for CGS: H[pass][i] = sum of partials i
__global__ void __launch_bounds__(256) k_reduce_multi(const int* __restrict__ off, int count,
                                                      const int* __restrict__ active,
                                                      const double* __restrict__ partial, int j, int pass, Scal* Sc) {
  const int inst = blockIdx.x;
  if (inst >= count) return;
  if (active && !active[inst]) return;
  if (j < 0) j = Sc[inst].j;
  const int b0 = off[inst], b1 = off[inst + 1];
  for (int i = 0; i <= j; ++i) {
    double acc = 0.0;
    for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
      acc += partial[(long long)b * (PCB_MAX_RESTART + 1) + i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) Sc[inst].H[pass * (PCB_MAX_RESTART + 1) + i] = s;
  }
}

// swap slot pointers (per instance, one thread)
__global__ void k_swap(Slots* S, int count, const int* __restrict__ active, int a0, int b0, int a1, int b1, int a2,
                       int b2) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= count) return;
  if (active && !active[inst]) return;
  double* t;
  if (a0 >= 0) { t = S[inst].v[a0]; S[inst].v[a0] = S[inst].v[b0]; S[inst].v[b0] = t; }
  if (a1 >= 0) { t = S[inst].v[a1]; S[inst].v[a1] = S[inst].v[b1]; S[inst].v[b1] = t; }
  if (a2 >= 0) { t = S[inst].v[a2]; S[inst].v[a2] = S[inst].v[b2]; S[inst].v[b2] = t; }
}

// set slot `dst` = slot `base` + k * 2mn  (GMRES basis addressing); per_j: k is an offset from
// the instance's own Arnoldi index
__global__ void k_setslot(const Geom* __restrict__ G, Slots* S, const Scal* __restrict__ Sc, int count,
                          const int* __restrict__ active, int dst, int base, int k, int per_j) {
  const int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= count) return;
  if (active && !active[inst]) return;
  const int kk = per_j ? Sc[inst].j + k : k;
  S[inst].v[dst] = S[inst].v[base] + (long long)kk * 2 * G[inst].mn;
}

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
cudaError_t launch_dot(const Batch& B, int sa, int sb) {
  k_dot<<<B.tot_vec, 256, 0, B.stream>>>(B.G, B.S, B.off_vec, B.count, B.active, sa, sb, B.partial);
  return cudaGetLastError();
}
cudaError_t launch_reduce(const Batch& B, const int* off, int nper, int which, int step, double tol, int j,
                          int restart) {
  k_reduce<<<B.count, 256, 0, B.stream>>>(off, B.count, B.active, B.partial, nper, which, B.Sc, step, tol, B.tols, j,
                                          restart);
  return cudaGetLastError();
}
cudaError_t launch_axpby(const Batch& B, int mode, int sx, int sy, int sz) {
  k_axpby<<<B.tot_vec, 256, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_vec, B.count, B.active, mode, sx, sy, sz);
  return cudaGetLastError();
}
cudaError_t launch_minres_wx(const Batch& B, int sy, int sw, int sw2, int sx) {
  k_minres_wx<<<B.tot_vec, 256, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_vec, B.count, B.active, sy, sw, sw2, sx);
  return cudaGetLastError();
}
// basis-loop bound for Arnoldi index j (j < 0: per-instance indices, at most jmax when jmax >= 0).
// The loops are unrolled to the bound and predicated beyond j + 1; the kernels are bound by FP64
// issue, so a predicated-off step still costs its slot: the bound is exact up to 20 basis vectors
// and a multiple of 4 above (most solves stay in the exact range).
static int basis_bound(int j, int jmax) {
  if (j < 0) j = jmax;
  const int need = j < 0 ? PCB_MAX_RESTART + 1 : j + 1;
  if (need <= 20) return need < 1 ? 1 : need;
  return need <= 24 ? 24 : need <= 28 ? 28 : PCB_MAX_RESTART + 1;
}
#define PCB_BASIS_BOUNDS(X)                                                                           \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) \
  X(19) X(20) X(24) X(28)
cudaError_t launch_multidot(const Batch& B, int svbase, int j, int sw, int jmax) {
#define PCB_MULTIDOT(JB) \
  k_multidot<JB><<<B.tot_vec, 256, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_vec, B.count, B.active, svbase, j, sw, B.partial)
#define PCB_MULTIDOT_CASE(JB) case JB: PCB_MULTIDOT(JB); break;
  switch (basis_bound(j, jmax)) {
    PCB_BASIS_BOUNDS(PCB_MULTIDOT_CASE)
    default: PCB_MULTIDOT(PCB_MAX_RESTART + 1); break;
  }
#undef PCB_MULTIDOT_CASE
#undef PCB_MULTIDOT
  return cudaGetLastError();
}
cudaError_t launch_reduce_multi(const Batch& B, int j, int pass) {
  k_reduce_multi<<<B.count, 256, 0, B.stream>>>(B.off_vec, B.count, B.active, B.partial, j, pass, B.Sc);
  return cudaGetLastError();
}
cudaError_t launch_multiaxpy(const Batch& B, int svbase, int j, int sw, int pass, int jmax) {
#define PCB_MULTIAXPY(JB) \
  k_multiaxpy<JB><<<B.tot_vec, 256, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_vec, B.count, B.active, svbase, j, sw, pass)
#define PCB_MULTIAXPY_CASE(JB) case JB: PCB_MULTIAXPY(JB); break;
  switch (basis_bound(j, jmax)) {
    PCB_BASIS_BOUNDS(PCB_MULTIAXPY_CASE)
    default: PCB_MULTIAXPY(PCB_MAX_RESTART + 1); break;
  }
#undef PCB_MULTIAXPY_CASE
#undef PCB_MULTIAXPY
  return cudaGetLastError();
}
cudaError_t launch_swap(const Batch& B, int a0, int b0, int a1, int b1, int a2, int b2) {
  k_swap<<<(B.count + 63) / 64, 64, 0, B.stream>>>(B.S, B.count, B.active, a0, b0, a1, b1, a2, b2);
  return cudaGetLastError();
}
cudaError_t launch_setslot(const Batch& B, int dst, int base, int k, int per_j) {
  k_setslot<<<(B.count + 63) / 64, 64, 0, B.stream>>>(B.G, B.S, B.Sc, B.count, B.active, dst, base, k, per_j);
  return cudaGetLastError();
}

}  // namespace pcb
