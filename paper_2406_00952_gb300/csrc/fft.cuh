// Shared-memory mixed-radix Stockham FFT over a set of lines held by one thread block.
//
// Each stage of radix R with `Ns` = product of the radices of the stages before it maps
// butterfly j (0 <= j < M/R) of a line to
//     inputs  in[j + r*M/R],  r = 0..R-1,  twiddled by w^(r*k), w = exp(-+2 pi i / (Ns R)), k = j mod Ns,
//     an R-point DFT,
//     outputs out[(j/Ns)*Ns*R + k + q*Ns], q = 0..R-1,
// which leaves the transform in natural order after the last stage (the autosort property),
// so stages ping-pong between two buffers and no bit reversal is needed.
// Forward uses exp(-2 pi i jk/M) with no scaling; inverse uses the conjugate twiddles, also
// unscaled.
#pragma once
#include "pcb_internal.cuh"

namespace pcb {

template <typename T>
__device__ __forceinline__ void dft2(T* a) {
  T t0 = cadd(a[0], a[1]);
  a[1] = csub(a[0], a[1]);
  a[0] = t0;
}

template <typename T>
__device__ __forceinline__ void dft4(T* a, bool inv) {
  T t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  T t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
  t3 = inv ? cmul_pi(t3) : cmul_mi(t3);
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}

template <typename T, typename R>
__device__ __forceinline__ void dft3(T* a, bool inv) {
  const R s = (R)0.86602540378443864676;   // sin(pi/3)
  T t1 = cadd(a[1], a[2]);
  T t2 = csub(a[1], a[2]);
  T m1 = csub(a[0], cscale(t1, (R)0.5));
  // forward: b1 = m1 - i s t2, b2 = m1 + i s t2 ; inverse swaps the sign
  T st = cscale(t2, s);
  T ist = inv ? cmul_pi(st) : cmul_mi(st);   // -i s t2 (forward)
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m1, ist);
  a[2] = csub(m1, ist);
}

template <typename T, typename R>
__device__ __forceinline__ void dft8(T* a, bool inv) {
  T e[4] = {a[0], a[2], a[4], a[6]};
  T o[4] = {a[1], a[3], a[5], a[7]};
  dft4(e, inv);
  dft4(o, inv);
  const R r = (R)0.70710678118654752440;
  // w8^k o_k, w8 = exp(-+ i pi / 4)
  T w1 = mk<R>(r, inv ? r : -r);
  T w3 = mk<R>(-r, inv ? r : -r);
  o[1] = cmul(o[1], w1);
  o[2] = inv ? cmul_pi(o[2]) : cmul_mi(o[2]);
  o[3] = cmul(o[3], w3);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = cadd(e[k], o[k]);
    a[k + 4] = csub(e[k], o[k]);
  }
}

template <typename R, int RAD>
__device__ __forceinline__ void stockham_stage(const cx<R>* __restrict__ in, cx<R>* __restrict__ out, int M, int Ns,
                                               int nlines, int ls, const cx<R>* __restrict__ tw, bool inv) {
  using T = cx<R>;
  const int nb = M / RAD;
  const int total = nb * nlines;
  const int step = M / (Ns * RAD);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = b / nb;
    const int j = b - line * nb;
    const T* src = in + line * ls;
    T* dst = out + line * ls;
    const int k = j % Ns;
    T a[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) a[r] = src[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        T w = tw[r * k * step];           // r*k*step < RAD*Ns*step = M
        if (inv) w.y = -w.y;
        a[r] = cmul(a[r], w);
      }
    }
    if (RAD == 2) dft2(a);
    else if (RAD == 3) dft3<T, R>(a, inv);
    else if (RAD == 4) dft4(a, inv);
    else dft8<T, R>(a, inv);
    const int base = (j / Ns) * Ns * RAD + k;
#pragma unroll
    for (int q = 0; q < RAD; ++q) dst[base + q * Ns] = a[q];
  }
}

// Transform `nlines` lines (line l at buf0 + l*ls, length plan.M) in place from buf0's point of
// view: returns the buffer (buf0 or buf1) that holds the result.  Must be called by all threads
// of the block; synchronises before returning.
template <typename R>
__device__ cx<R>* fft_lines(cx<R>* buf0, cx<R>* buf1, const FftPlan& plan, int nlines, int ls,
                            const cx<R>* __restrict__ tw, bool inv) {
  cx<R>* in = buf0;
  cx<R>* out = buf1;
  int Ns = 1;
  for (int s = 0; s < plan.nst; ++s) {
    const int rad = plan.rad[s];
    switch (rad) {
      case 2: stockham_stage<R, 2>(in, out, plan.M, Ns, nlines, ls, tw, inv); break;
      case 3: stockham_stage<R, 3>(in, out, plan.M, Ns, nlines, ls, tw, inv); break;
      case 4: stockham_stage<R, 4>(in, out, plan.M, Ns, nlines, ls, tw, inv); break;
      default: stockham_stage<R, 8>(in, out, plan.M, Ns, nlines, ls, tw, inv); break;
    }
    Ns *= rad;
    __syncthreads();
    cx<R>* t = in; in = out; out = t;
  }
  return in;
}

}  // namespace pcb
