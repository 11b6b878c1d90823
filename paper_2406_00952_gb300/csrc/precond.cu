// Preconditioner applications |P_S|^{-1}, P_S^{-1} and P_MS^{-1} for a(x) = 1 (paper Sec. 3.5).
//
// With Q = (F D* (x) S_N (x) S_N) (time DFT after the zeta = pi scaling, 2D DST-I in space),
// |P_S|, P_S and P_MS are block diagonal in Q's basis (Sec. 3.5, three-step applications), so
//     P^{-1} v = Q^{-1} (pointwise solve) Q v.
// The transforms along the three axes commute, so the apply runs as five batched passes, each
// along one full axis inside shared memory:
//     DST along x1  ->  DST along x2  ->  [time DFT, pointwise solve, inverse time DFT]
//     ->  DST along x2  ->  DST along x1.
// The spatial passes keep the data real: the two halves (y~ and p~ blocks) of the all-at-once
// vector ride as real and imaginary parts of one complex line, and the DST-I of order L = N+1
// comes from the length-2L FFT of the odd extension (Y_p = -2i * DST(x)_p).
// The time pass packs the two halves the same way; for zeta = pi the F-slot r of a real series
// and slot n-1-r are complex conjugates, which separates the halves per frequency pair.
#include "fft.cuh"

namespace pcb {

enum { PK_ABS_PS = 1, PK_PS = 2, PK_PMS = 3 };

template <typename R> __device__ __forceinline__ const cx<R>* twd(const Geom& g);
template <> __device__ __forceinline__ const float2* twd<float>(const Geom& g) { return g.twd_f; }
template <> __device__ __forceinline__ const double2* twd<double>(const Geom& g) { return g.twd_d; }
template <typename R> __device__ __forceinline__ const cx<R>* twt(const Geom& g);
template <> __device__ __forceinline__ const float2* twt<float>(const Geom& g) { return g.twt_f; }
template <> __device__ __forceinline__ const double2* twt<double>(const Geom& g) { return g.twt_d; }
template <typename R> __device__ __forceinline__ const cx<R>* pre(const Geom& g);
template <> __device__ __forceinline__ const float2* pre<float>(const Geom& g) { return g.pre_f; }
template <> __device__ __forceinline__ const double2* pre<double>(const Geom& g) { return g.pre_d; }
template <typename R> __device__ __forceinline__ const cx<R>* mutab(const Geom& g);
template <> __device__ __forceinline__ const float2* mutab<float>(const Geom& g) { return g.mu_f; }
template <> __device__ __forceinline__ const double2* mutab<double>(const Geom& g) { return g.mu_d; }

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }

// ------------------------------------------------------------------------------------------
// DST-I pass along x1 (axis 0) or x2 (axis 1), both halves at once.
// in_slot / out_slot >= 0 select a vector slot (FP64), -1 selects the instance scratch (R).
// ------------------------------------------------------------------------------------------
template <typename TIn, typename TOut, typename R>
__global__ void __launch_bounds__(256) k_dst(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                             const int* __restrict__ off, int count,
                                             const int* __restrict__ active, int axis, int in_slot,
                                             int out_slot) {
  using T = cx<R>;
  const int inst = find_inst(off, count, blockIdx.x);
  if (active && !active[inst]) return;
  const Geom& g = G[inst];
  const int lb = blockIdx.x - off[inst];
  const TIn* __restrict__ in = in_slot >= 0 ? (const TIn*)S[inst].v[in_slot] : (const TIn*)g.scratch;
  TOut* __restrict__ out = out_slot >= 0 ? (TOut*)S[inst].v[out_slot] : (TOut*)g.scratch;
  const int N = g.N, M = g.M, L = g.L, lpb = g.dst_lpb[sizeof(R) == 4], ls = M + 1;
  const long long mn = g.mn;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* b0 = (T*)smem_raw;
  T* b1 = b0 + lpb * ls;

  long long line0 = 0;
  int t = 0, i0 = 0;
  if (axis == 0) {
    line0 = (long long)lb * lpb;
  } else {
    const int nbt = (N + lpb - 1) / lpb;
    t = lb / nbt;
    i0 = (lb - t * nbt) * lpb;
  }
  const long long nlines0 = (long long)g.n * N;
  const int tot = lpb * N;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int l, q;
    long long addr;
    bool valid;
    if (axis == 0) {
      l = e / N; q = e - l * N;
      const long long line = line0 + l;
      valid = line < nlines0;
      addr = line * N + q;
    } else {
      q = e / lpb; l = e - q * lpb;
      const int i = i0 + l;
      valid = i < N;
      addr = (long long)t * g.m + (long long)q * N + i;
    }
    R v0 = 0, v1 = 0;
    if (valid) { v0 = (R)in[addr]; v1 = (R)in[mn + addr]; }
    b0[l * ls + q + 1] = mk<R>(v0, v1);
    b0[l * ls + M - q - 1] = mk<R>(-v0, -v1);
  }
  for (int l = threadIdx.x; l < lpb; l += blockDim.x) {
    b0[l * ls] = mk<R>(0, 0);
    b0[l * ls + L] = mk<R>(0, 0);
  }
  __syncthreads();
  const T* res = fft_lines<R>(b0, b1, g.pdst, lpb, ls, twd<R>(g), false);
  const R s = (R)(0.5 * sqrt(2.0 / (double)L));
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    int l, q;
    long long addr;
    bool valid;
    if (axis == 0) {
      l = e / N; q = e - l * N;
      const long long line = line0 + l;
      valid = line < nlines0;
      addr = line * N + q;
    } else {
      q = e / lpb; l = e - q * lpb;
      const int i = i0 + l;
      valid = i < N;
      addr = (long long)t * g.m + (long long)q * N + i;
    }
    if (valid) {
      const T Y = res[l * ls + q + 1];
      out[addr] = (TOut)(-Y.y * s);
      out[mn + addr] = (TOut)(Y.x * s);
    }
  }
}

// ------------------------------------------------------------------------------------------
// Time pass: forward DFT of (half0 + i half1) * exp(-i pi t/n), pointwise solve per frequency
// pair, inverse DFT, unscale.  In place on the scratch.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_time(const Geom* __restrict__ G, const int* __restrict__ off, int count,
                                              const int* __restrict__ active, int kind) {
  using T = cx<R>;
  const int inst = find_inst(off, count, blockIdx.x);
  if (active && !active[inst]) return;
  const Geom& g = G[inst];
  const int lb = blockIdx.x - off[inst];
  R* __restrict__ y = (R*)g.scratch;
  const int n = g.n, m = g.m, N = g.N, cpb = g.time_cpb[sizeof(R) == 4], ls = n + 1;
  const long long mn = g.mn;
  const int c0 = lb * cpb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* b0 = (T*)smem_raw;
  T* b1 = b0 + cpb * ls;
  const T* __restrict__ pr = pre<R>(g);

  const int tot = cpb * n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int tt = e / cpb, l = e - tt * cpb;
    const int col = c0 + l;
    T v = mk<R>(0, 0);
    if (col < m) {
      const long long a = (long long)tt * m + col;
      v = cmul(mk<R>(y[a], y[mn + a]), pr[tt]);
    }
    b0[l * ls + tt] = v;
  }
  __syncthreads();
  T* f = fft_lines<R>(b0, b1, g.ptime, cpb, ls, twt<R>(g), false);
  T* other = (f == b0) ? b1 : b0;

  const T* __restrict__ mu = mutab<R>(g);
  const R alpha = (R)g.alpha, a2 = (R)(g.alpha * g.alpha);
  const int half = n / 2;
  const int totp = cpb * half;
  for (int e = threadIdx.x; e < totp; e += blockDim.x) {
    const int l = e / half, r = e - l * half;
    const int col = c0 + l;
    if (col >= m) continue;
    const int j = col / N, i = col - j * N;
    const R c = (R)(g.tau * (g.kap[i] + g.kap[j]));
    const int rp = n - 1 - r;
    T* line = f + l * ls;
    const T mr = mu[r];
    const T lam = mk<R>(mr.x + c, mr.y);
    const R mod2 = lam.x * lam.x + lam.y * lam.y;
    if (kind == PK_ABS_PS) {
      const R w = rsqrt_<R>(mod2 + a2);
      line[r] = cscale(line[r], w);
      line[rp] = cscale(line[rp], w);
    } else if (kind == PK_PMS) {
      const R sig = sqrt(mr.x * mr.x + mr.y * mr.y + a2);
      const R w = (R)1 / (sig + c);
      line[r] = cscale(line[r], w);
      line[rp] = cscale(line[rp], w);
    } else {
      const T Cr = line[r], Cq = cconj(line[rp]);
      const T F1 = cscale(cadd(Cr, Cq), (R)0.5);
      const T F2 = cmul_mi(cscale(csub(Cr, Cq), (R)0.5));
      const R inv = (R)1 / (mod2 + a2);
      // U1 = (conj(lam) F1 + alpha F2)/det, U2 = (lam F2 - alpha F1)/det
      const T U1 = cscale(cadd(cmul(cconj(lam), F1), cscale(F2, alpha)), inv);
      const T U2 = cscale(csub(cmul(lam, F2), cscale(F1, alpha)), inv);
      line[r] = cadd(U1, cmul_pi(U2));
      line[rp] = cadd(cconj(U1), cmul_pi(cconj(U2)));
    }
  }
  __syncthreads();
  T* res = fft_lines<R>(f, other, g.ptime, cpb, ls, twt<R>(g), true);
  const R sc = (R)1 / (R)n;
  for (int e = threadIdx.x; e < tot; e += blockDim.x) {
    const int tt = e / cpb, l = e - tt * cpb;
    const int col = c0 + l;
    if (col < m) {
      const T v = cscale(cmul(res[l * ls + tt], cconj(pr[tt])), sc);
      const long long a = (long long)tt * m + col;
      y[a] = v.x;
      y[mn + a] = v.y;
    }
  }
}

// ------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------
template <typename R>
static size_t dst_smem(const Batch& B) { return (size_t)2 * B.max_lpb_M[sizeof(R) == 4] * sizeof(cx<R>); }
template <typename R>
static size_t time_smem(const Batch& B) { return (size_t)2 * B.max_cpb_n[sizeof(R) == 4] * sizeof(cx<R>); }

template <typename R>
static cudaError_t precond_passes(const Batch& B, int kind, int in_slot, int out_slot) {
  const size_t sd = dst_smem<R>(B), st = time_smem<R>(B);
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_dst<double, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_dst<R, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_dst<R, double, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_time<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_done = true;
  }
  const int p = sizeof(R) == 4;
  k_dst<double, R, R><<<B.tot_dst_i[p], 256, sd, B.stream>>>(B.G, B.S, B.off_dst_i[p], B.count, B.active, 0, in_slot, -1);
  k_dst<R, R, R><<<B.tot_dst_j[p], 256, sd, B.stream>>>(B.G, B.S, B.off_dst_j[p], B.count, B.active, 1, -1, -1);
  k_time<R><<<B.tot_time[p], 256, st, B.stream>>>(B.G, B.off_time[p], B.count, B.active, kind);
  k_dst<R, R, R><<<B.tot_dst_j[p], 256, sd, B.stream>>>(B.G, B.S, B.off_dst_j[p], B.count, B.active, 1, -1, -1);
  k_dst<R, double, R><<<B.tot_dst_i[p], 256, sd, B.stream>>>(B.G, B.S, B.off_dst_i[p], B.count, B.active, 0, -1, out_slot);
  return cudaGetLastError();
}

cudaError_t launch_precond_fast(const Batch& B, int kind, int prec, int in_slot, int out_slot) {
  return prec == PCB_MIXED ? precond_passes<float>(B, kind, in_slot, out_slot)
                           : precond_passes<double>(B, kind, in_slot, out_slot);
}

}  // namespace pcb
