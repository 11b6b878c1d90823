// Register / warp-shuffle FFTs for lines of length M = P * Q (P lanes of a warp, Q values per lane).
//
// Lane t of a P-lane group holds x[t + P q], q = 0..Q-1 (consecutive lanes hold consecutive
// elements, so loads from a contiguous line are conflict-free).  With s = t + P q and
// k = k1 + Q k2:
//     X[k1 + Q k2] = sum_t W_P^{t k2} W_M^{t k1} sum_q x[t + P q] W_Q^{q k1}
// so each lane runs a Q-point DFT in registers, multiplies by W_M^{t k1}, and the P-point DFTs
// over t run as radix-2 decimation-in-frequency stages across lanes (__shfl_xor), leaving
// lane t with X[k1 + Q bitrev_P(t)].  Forward uses W = exp(-2 pi i / M); inverse conjugates.
#pragma once
#include <math.h>

#include "pcb_internal.cuh"

namespace pcb {

// W_96^k = exp(-2 pi i k / 96): covers every twiddle of the register DFTs (Q | 96) and of the
// cross-lane stages (2d | 32).  One copy per translation unit that includes this header; each
// such unit fills its copy with upload_w96() before its first launch.
static __constant__ float2 c_w96f[96];
static __constant__ double2 c_w96d[96];

static cudaError_t upload_w96() {
  float2 f[96];
  double2 d[96];
  for (int k = 0; k < 96; ++k) {
    const double a = -2.0 * 3.14159265358979323846 * k / 96.0;
    d[k].x = cos(a); d[k].y = sin(a);
    f[k].x = (float)d[k].x; f[k].y = (float)d[k].y;
  }
  cudaError_t e = cudaMemcpyToSymbol(c_w96f, f, sizeof(f));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_w96d, d, sizeof(d));
}

template <typename R> __device__ __forceinline__ cx<R> w96(int k);
template <> __device__ __forceinline__ float2 w96<float>(int k) { return c_w96f[k]; }
template <> __device__ __forceinline__ double2 w96<double>(int k) { return c_w96d[k]; }

template <typename T>
__device__ __forceinline__ void r2(T& a, T& b) { T t = cadd(a, b); b = csub(a, b); a = t; }

template <typename T>
__device__ __forceinline__ void r4(T* a, bool inv) {
  T t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  T t2 = cadd(a[1], a[3]), t3 = csub(a[1], a[3]);
  t3 = inv ? cmul_pi(t3) : cmul_mi(t3);
  a[0] = cadd(t0, t2); a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3); a[3] = csub(t1, t3);
}

template <typename T, typename R>
__device__ __forceinline__ void r3(T* a, bool inv) {
  const R s = (R)0.86602540378443864676;
  T t1 = cadd(a[1], a[2]), t2 = csub(a[1], a[2]);
  T m1 = csub(a[0], cscale(t1, (R)0.5));
  T st = cscale(t2, s);
  T ist = inv ? cmul_pi(st) : cmul_mi(st);
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m1, ist);
  a[2] = csub(m1, ist);
}

template <typename T, typename R>
__device__ __forceinline__ void r8(T* a, bool inv) {
  T e[4] = {a[0], a[2], a[4], a[6]};
  T o[4] = {a[1], a[3], a[5], a[7]};
  r4(e, inv); r4(o, inv);
  const R h = (R)0.70710678118654752440;
  o[1] = cmul(o[1], mk<R>(h, inv ? h : -h));
  o[2] = inv ? cmul_pi(o[2]) : cmul_mi(o[2]);
  o[3] = cmul(o[3], mk<R>(-h, inv ? h : -h));
#pragma unroll
  for (int k = 0; k < 4; ++k) { a[k] = cadd(e[k], o[k]); a[k + 4] = csub(e[k], o[k]); }
}

// Primitive DFT of size Q on x[0..Q) in place, natural output order.
template <typename T, typename R, int Q>
__device__ __forceinline__ void prim(T* x, bool inv) {
  if (Q == 2) r2(x[0], x[1]);
  else if (Q == 3) r3<T, R>(x, inv);
  else if (Q == 4) r4(x, inv);
  else if (Q == 8) r8<T, R>(x, inv);
}

// Register DFT of size Q = A*B (A, B primitive) or primitive Q.  Output X[k] is left in
// register pos<Q>(k): identity for primitive sizes, (k / A) + B * (k % A) for composites.
template <int Q> struct Split { static constexpr int A = Q, B = 1; };
template <> struct Split<6> { static constexpr int A = 2, B = 3; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };
template <> struct Split<24> { static constexpr int A = 8, B = 3; };
template <> struct Split<32> { static constexpr int A = 4, B = 8; };

template <int Q> __device__ __forceinline__ constexpr int pos(int k) {
  return Split<Q>::B == 1 ? k : (k / Split<Q>::A) + Split<Q>::B * (k % Split<Q>::A);
}

template <typename T, typename R, int Q>
__device__ __forceinline__ void reg_dft(T* x, bool inv) {
  constexpr int A = Split<Q>::A, B = Split<Q>::B;
  if constexpr (B == 1) {
    prim<T, R, Q>(x, inv);
  } else {
  // step 1: for each b, A-point DFT over x[b + B a]; result Y_b[k1] stays at x[b + B k1]
#pragma unroll
  for (int b = 0; b < B; ++b) {
    T t[A > 1 ? A : 1];
#pragma unroll
    for (int a = 0; a < A; ++a) t[a] = x[b + B * a];
    prim<T, R, A>(t, inv);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      T v = t[k1];
      if (b * k1) {
        T w = w96<R>((b * k1 * (96 / Q)) % 96);
        if (inv) w.y = -w.y;
        v = cmul(v, w);
      }
      x[b + B * k1] = v;
    }
  }
  // step 2: for each k1, B-point DFT over the contiguous chunk x[B k1 .. B k1 + B)
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) prim<T, R, B>(x + B * k1, inv);
  }
}

// Cross-lane radix-2 DIF over P lanes (P a power of two <= 32) for each of the Q registers.
// Stage s (half-width d = P >> (s+1)): lower lanes keep v + u, upper lanes (u - v) W_{2d}^{t mod d}.
// Written as (u + sg*v) * we with sg = +-1 and we = 1 or the twiddle, so every lane runs the
// same instruction stream (no select).
template <typename T, typename R>
struct LaneStages {
  T we[5];
  R sg[5];
  int n;
};

template <typename T, typename R>
__device__ __forceinline__ void lane_stages(LaneStages<T, R>& st, int t, int P, bool inv) {
  const int nst = __ffs(P) - 1;   // log2 P
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    st.we[s] = mk<R>((R)1, (R)0);
    st.sg[s] = (R)1;
    if (s < nst) {
      const int d = P >> (s + 1);
      const bool upper = (t & d) != 0;
      T w = w96<R>(((t & (d - 1)) * (96 / (2 * d))) % 96);
      if (inv) w.y = -w.y;
      if (upper) { st.we[s] = w; st.sg[s] = (R)-1; }
    }
  }
  st.n = nst;
}

template <typename T, typename R, int Q>
__device__ __forceinline__ void lane_dif(T* x, int P, const LaneStages<T, R>& st) {
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    if (s >= st.n) break;
    const int d = P >> (s + 1);
    const T w = st.we[s];
    const R sg = st.sg[s];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const T v = x[q];
      T a;
      a.x = __shfl_xor_sync(0xffffffffu, v.x, d);
      a.y = __shfl_xor_sync(0xffffffffu, v.y, d);
      x[q] = cmul(cfma_s(sg, v, a), w);
    }
  }
}

__device__ __forceinline__ int bitrev(int t, int P) {
  return P <= 1 ? 0 : (int)(__brev((unsigned)t) >> (32 - __ffs(P) + 1));
}

// padded shared-memory index: one gap every 32 elements
__device__ __forceinline__ int pidx(int s) { return s + (s >> 5); }

}  // namespace pcb
