// Preconditioner applications |P_S|^{-1}, P_S^{-1} and P_MS^{-1} for a(x) = 1 (paper Sec. 3.5).
//
// With Q = (F D* (x) S_N (x) S_N) (time DFT after the zeta = pi scaling, 2D DST-I in space),
// |P_S|, P_S and P_MS are block diagonal in Q's basis (Sec. 3.5, three-step applications), so
//     P^{-1} v = Q^{-1} (pointwise solve) Q v.
// The transforms along the three axes commute, so the apply runs as five batched passes, each
// along one full axis:
//     DST along x1  ->  DST along x2  ->  [time DFT, pointwise solve, inverse time DFT]
//     ->  DST along x2  ->  DST along x1.
// The spatial passes keep the data real: the two halves (y~ and p~ blocks) of the all-at-once
// vector ride as real and imaginary parts of one complex line, and the DST-I of order L = N+1
// comes from the length-2L FFT of the odd extension (Y_p = -2i * DST(x)_p).
// The time pass packs the two halves the same way; for zeta = pi the F-slot r of a real series
// and slot n-1-r are complex conjugates, which separates the halves per frequency pair (other
// zeta: time_body_general, two complex lines per point).  Neumann problems (Example 3) take the
// scaled DCT-I pair of order L = N-1 from the even extension in the same spatial passes.
//
// Each pass stages a tile of lines through padded shared memory (coalesced global access in both
// directions); each line is transformed by a group of P <= 32 lanes holding Q values each
// (register DFT + warp-shuffle stages, fft_reg.cuh).
#include <algorithm>

#include "fft_reg.cuh"

namespace pcb {

enum { PK_ABS_PS = 1, PK_PS = 2, PK_PMS = 3 };
int mg_launch_count(int kind);

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

// padded line length (in complex elements) able to hold indices 0..len-1 under pidx(), odd so
// that consecutive lines start in different banks
__host__ __device__ __forceinline__ int padded_len(int len) { return (len + (len >> 5) + 1) | 1; }

// ------------------------------------------------------------------------------------------
// Line transform shared by the passes.  On entry lane t of a P-lane group has x[q] = element
// t + P q of its line.  Afterwards the lane owns Q transform values; owned(j) gives the output
// index of the j-th one and value(j) its register.
//   Q < 32 : register DFT, twiddle, cross-lane DIF; owned(j) = j + Q bitrev_P(t).
//   Q = 32 (P = 32): register DFT, twiddle, transpose through the warp's 32 x 33 scratch,
//            second 32-point register DFT; owned(j) = t + 32 j (natural, lane-strided order).
// ------------------------------------------------------------------------------------------
template <typename T, typename R, int Q>
struct LineFFT {
  T x[Q];
  __device__ __forceinline__ void run(int t, int P, const LaneStages<T, R>& st, const T* __restrict__ tw,
                                      const T* twq, T* scratch, bool inv) {
    reg_dft<T, R, Q>(x, inv);
    if constexpr (Q == 32) {
      // twiddle and transpose-store in groups of eight; the empty asm with a memory clobber keeps
      // the compiler from hoisting all 31 twiddle loads (register pressure)
#pragma unroll
      for (int g8 = 0; g8 < 4; ++g8) {
        T w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = __ldg(&tw[t * (g8 * 8 + u)]);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k1 = g8 * 8 + u;
          T v = x[pos<32>(k1)];
          if (k1) { T ww = w[u]; if (inv) ww.y = -ww.y; v = cmul(v, ww); }
          scratch[k1 * 33 + t] = v;
        }
        asm volatile("" ::: "memory");
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 32; ++u) x[u] = scratch[t * 33 + u];
      __syncwarp();
      reg_dft<T, R, 32>(x, inv);
    } else {
#pragma unroll
      for (int k1 = 1; k1 < Q; ++k1) {
        T w = twq[k1];
        if (inv) w.y = -w.y;
        x[pos<Q>(k1)] = cmul(x[pos<Q>(k1)], w);
      }
      lane_dif<T, R, Q>(x, P, st);
    }
  }
  __device__ __forceinline__ static int owned(int j, int t, int k2) { return Q == 32 ? t + 32 * j : j + Q * k2; }
  __device__ __forceinline__ T value(int j) const { return x[pos<Q>(j)]; }
};

// ------------------------------------------------------------------------------------------
// Spatial pass along x1 (axis 0) or x2 (axis 1), both halves at once: the orthonormal DST-I of
// order L = N+1 (Dirichlet), or for Neumann the scaled DCT-I pair of order L = N-1, forward
// (inv = 0: u -> C W^{1/2} u) or inverse (inv = 1: v -> W^{-1/2} C v), with C the orthonormal
// DCT-I and W = diag(1/2, 1, .., 1, 1/2).  Both come from one length-2L FFT of the line's
// extension: odd (Y_p = -2i DST(x)_p) or even (Y_k = 2 sum_i w_i x_i cos(pi i k / L)).
// in_slot / out_slot >= 0 select a vector slot (FP64), -1 selects the instance scratch (R).
// ------------------------------------------------------------------------------------------
template <typename TIn, typename TOut, typename R, int Q>
__device__ __forceinline__ void dst_body(const Geom& g, const Slots* __restrict__ S, int inst, int lb, int axis,
                                         int in_slot, int out_slot, int inv) {
  using T = cx<R>;
  const TIn* __restrict__ in = in_slot >= 0 ? (const TIn*)S[inst].v[in_slot] : (const TIn*)g.scratch;
  TOut* __restrict__ out = out_slot >= 0 ? (TOut*)S[inst].v[out_slot] : (TOut*)g.scratch;
  const int N = g.N, L = g.L, M = g.M;
  const bool neu = g.bc == PCB_BC_NEUMANN;
  const int lpb = axis == 0 ? g.dst_lpb[sizeof(R) == 4] : g.dst_lpb_j[sizeof(R) == 4];   // power of two
  const int ls = padded_len(N + 1);          // element q of a line at padded index q + 1
  const long long mn = g.mn;
  const int m = g.m;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = (T*)smem_raw;
  const int nthr = blockDim.x, tid = threadIdx.x;

  long long line0 = 0;
  int t0 = 0, i0 = 0;
  if (axis == 0) {
    line0 = (long long)lb * lpb;
  } else {
    const int nbt = (N + lpb - 1) / lpb;
    t0 = lb / nbt;
    i0 = (lb - t0 * nbt) * lpb;
  }
  const long long nlines0 = (long long)g.n * N;
  const int lsh = __ffs(lpb) - 1;
  // ---- load tile: line l, element q (0-based) at padded index q+1.  Each thread walks the
  // flattened tile with incremental indices and issues eight independent loads per step.
  if (axis == 0) {
    const long long nval = (nlines0 - line0) * N;        // valid elements from line0 on
    const int tot = lpb * N;
    const TIn* src = in + line0 * N;
    int e = tid;
    int l = e / N, q = e - l * N;                          // one division per thread
    const int dl = nthr / N, dq = nthr - dl * N;
    for (; e < tot; ) {
      R v0[8], v1[8];
      int ls_[8], qs_[8];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (e < tot) {
          const bool ok = e < nval;
          v0[u] = ok ? (R)src[e] : (R)0;
          v1[u] = ok ? (R)src[mn + e] : (R)0;
          ls_[u] = l; qs_[u] = q;
          ++cnt;
          e += nthr; l += dl; q += dq;
          if (q >= N) { q -= N; ++l; }
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (u < cnt) tile[ls_[u] * ls + pidx(qs_[u] + 1)] = mk<R>(v0[u], v1[u]);
    }
  } else {
    const int l = tid & (lpb - 1), qs = nthr >> lsh;
    const int i = i0 + l;
    const TIn* src = in + (long long)t0 * m + i;
    T* dst = tile + l * ls;
    const bool iv = i < N;
    for (int q = tid >> lsh; q < N; q += 8 * qs) {
      R v0[8], v1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int qq = q + u * qs;
        const bool ok = iv && qq < N;
        v0[u] = ok ? (R)src[(long long)qq * N] : (R)0;
        v1[u] = ok ? (R)src[mn + (long long)qq * N] : (R)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int qq = q + u * qs;
        if (qq < N) dst[pidx(qq + 1)] = mk<R>(v0[u], v1[u]);
      }
    }
  }
  __syncthreads();
  // ---- transform: groups of P lanes, one line each
  const int P = M / Q;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int lpw = 32 / P;
  const int t = lane % P;
  LaneStages<T, R> st;
  lane_stages<T, R>(st, t, P, false);
  const T* __restrict__ tw = twd<R>(g);
  T twq[Q < 32 ? Q : 1];
  if constexpr (Q < 32) {
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) twq[k1] = __ldg(&tw[t * k1]);
  }
  T* wscr = tile + lpb * ls + warp * (32 * 33);
  const R sc = (R)(0.5 * sqrt(2.0 / (double)L));      // orthonormal scale of both DST-I and DCT-I
  const R rt2 = (R)1.4142135623730951, irt2 = (R)0.7071067811865476;
  const int k2 = bitrev(t, P);
  for (int lbase = warp * lpw; lbase < lpb; lbase += nw * lpw) {
    const int l = lbase + lane / P;
    const bool lv = l < lpb;
    T* line = tile + (lv ? l : 0) * ls;
    LineFFT<T, R, Q> f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = t + P * q;
      T v = mk<R>(0, 0);
      if (lv) {
        if (neu) {
          // even extension of element j = s (s <= L) or 2L - s; the inverse enters W^{-1/2} v
          const int j = s <= L ? s : M - s;
          v = line[pidx(j + 1)];
          if (inv && (j == 0 || j == L)) v = cscale(v, rt2);
        } else if (s > 0 && s < L) {
          v = line[pidx(s)];
        } else if (s > L) {
          v = line[pidx(M - s)]; v.x = -v.x; v.y = -v.y;
        }
      }
      f.x[q] = v;
    }
    f.run(t, P, st, tw, twq, wscr, false);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < Q; ++j) {
      const int p = LineFFT<T, R, Q>::owned(j, t, k2);
      if (neu) {
        // a real line's even extension has a real transform: both halves stay in place; the
        // forward pass applies W^{1/2} to the two end modes
        if (lv && p <= L) {
          const R fct = (!inv && (p == 0 || p == L)) ? sc * irt2 : sc;
          line[pidx(p + 1)] = cscale(f.value(j), fct);
        }
      } else if (lv && p >= 1 && p <= N) {
        const T Y = f.value(j);
        line[pidx(p)] = mk<R>(-Y.y * sc, Y.x * sc);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  // ---- store tile
  if (axis == 0) {
    for (int l = 0; l < lpb; ++l) {
      const long long line = line0 + l;
      if (line >= nlines0) break;
      const T* srcs = tile + l * ls;
      TOut* d = out + line * N;
      for (int q = tid; q < N; q += nthr) {
        const T Y = srcs[pidx(q + 1)];
        d[q] = (TOut)Y.x;
        d[mn + q] = (TOut)Y.y;
      }
    }
  } else {
    const int l = tid & (lpb - 1), qs = nthr >> lsh;
    const int i = i0 + l;
    if (i < N) {
      TOut* d = out + (long long)t0 * m + i;
      const T* srcs = tile + l * ls;
      for (int q = tid >> lsh; q < N; q += qs) {
        const T Y = srcs[pidx(q + 1)];
        d[(long long)q * N] = (TOut)Y.x;
        d[mn + (long long)q * N] = (TOut)Y.y;
      }
    }
  }
}

template <typename TIn, typename TOut, typename R, int Q>
__global__ void __launch_bounds__(256, 2) k_dst(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                             const int* __restrict__ off, int count,
                                             Sel sel, int axis, int in_slot,
                                             int out_slot, int inv) {
  const int inst = find_inst(off, count, blockIdx.x);
  if (sel.skip(inst)) return;
  dst_body<TIn, TOut, R, Q>(G[inst], S, inst, blockIdx.x - off[inst], axis, in_slot, out_slot, inv);
}

// Shared launch over instances with different line lengths: each block runs the register-FFT
// variant of its own instance.
template <typename TIn, typename TOut, typename R>
__global__ void __launch_bounds__(256, 2) k_dst_any(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                 const int* __restrict__ off, int count,
                                                 Sel sel, int axis, int in_slot,
                                                 int out_slot, int inv) {
  const int inst = find_inst(off, count, blockIdx.x);
  if (sel.skip(inst)) return;
  const Geom& g = G[inst];
  const int lb = blockIdx.x - off[inst];
  switch (g.dst_q) {
    case 1: dst_body<TIn, TOut, R, 1>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 2: dst_body<TIn, TOut, R, 2>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 3: dst_body<TIn, TOut, R, 3>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 4: dst_body<TIn, TOut, R, 4>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 6: dst_body<TIn, TOut, R, 6>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 8: dst_body<TIn, TOut, R, 8>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 12: dst_body<TIn, TOut, R, 12>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 16: dst_body<TIn, TOut, R, 16>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    case 24: dst_body<TIn, TOut, R, 24>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
    default: dst_body<TIn, TOut, R, 32>(g, S, inst, lb, axis, in_slot, out_slot, inv); break;
  }
}

// ------------------------------------------------------------------------------------------
// Time pass: forward DFT of (half0 + i half1) * exp(-i pi t/n), pointwise solve per frequency
// pair, inverse DFT, unscale.  In place on the scratch.
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// Time pass for a general zeta (omega = exp(i zeta), Sec. 3.5 with the circulant zeta = 0 and any
// other choice of Sec. 2).  Slot r of the DFT of x_t exp(-i zeta t/n) has frequency
// psi_r = -(zeta + 2 pi r)/n; unlike zeta = pi, the transform of a real series has no conjugate
// partner slot, so each half runs as its own complex line: forward DFT of v_h(t) exp(-i zeta t/n),
// the per-slot solve on (V_1, V_2) at each r, inverse DFT, unscale, real part (the operator
// applied to real vectors is Re(P^-1), symmetric positive definite for |P_S| and P_MS).
// ------------------------------------------------------------------------------------------
template <typename R, int Q>
__device__ __forceinline__ void time_body_general(const Geom& g, int lb, int kind) {
  using T = cx<R>;
  R* __restrict__ y = (R*)g.scratch;
  const int n = g.n, m = g.m, N = g.N, cpb = g.time_cpb[sizeof(R) == 4];
  const int ls = padded_len(n);
  const long long mn = g.mn;
  const int c0 = lb * cpb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = (T*)smem_raw;                        // line 2l + h: column c0 + l, half h
  const T* __restrict__ pr = pre<R>(g);
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int nl = 2 * cpb;
  for (int e = tid; e < cpb * n; e += nthr) {
    const int l = e % cpb, t = e / cpb;
    const int col = c0 + l;
    const bool cv = col < m;
    const long long a = (long long)t * m + (cv ? col : 0);
    const T w = __ldg(&pr[t]);
    const R v0 = cv ? y[a] : (R)0, v1 = cv ? y[mn + a] : (R)0;
    tile[(2 * l) * ls + pidx(t)] = mk<R>(v0 * w.x, v0 * w.y);
    tile[(2 * l + 1) * ls + pidx(t)] = mk<R>(v1 * w.x, v1 * w.y);
  }
  __syncthreads();
  const int P = n / Q;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int lpw = 32 / P;
  const int t = lane % P;
  const T* __restrict__ tw = twt<R>(g);
  T twq[Q < 32 ? Q : 1];
  if constexpr (Q < 32) {
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) twq[k1] = __ldg(&tw[t * k1]);
  }
  const int k2 = bitrev(t, P);
  for (int dir = 0; dir < 2; ++dir) {            // 0: forward, 1: inverse
    LaneStages<T, R> st;
    lane_stages<T, R>(st, t, P, dir == 1);
    for (int lbase = warp * lpw; lbase < nl; lbase += nw * lpw) {
      const int l = lbase + lane / P;
      const bool lv = l < nl;
      T* line = tile + (lv ? l : 0) * ls;
      LineFFT<T, R, Q> f;
#pragma unroll
      for (int q = 0; q < Q; ++q) f.x[q] = lv ? line[pidx(t + P * q)] : mk<R>(0, 0);
      __syncwarp();
      f.run(t, P, st, tw, twq, line, dir == 1);
      __syncwarp();
      if (lv) {
#pragma unroll
        for (int j = 0; j < Q; ++j) line[pidx(LineFFT<T, R, Q>::owned(j, t, k2))] = f.value(j);
      }
      __syncwarp();
    }
    __syncthreads();
    if (dir == 1) break;
    // per-slot solve of the pair (V_1, V_2) at slot r of column c0 + l
    const T* __restrict__ mu = mutab<R>(g);
    const R alpha = (R)g.alpha, a2 = (R)(g.alpha * g.alpha);
    for (int e = tid; e < cpb * n; e += nthr) {
      const int l = e / n, r = e - l * n;
      const int col = min(c0 + l, m - 1);
      const int jj = col / N, ii = col - jj * N;
      const R c = (R)(g.tau * (__ldg(&g.kap[ii]) + __ldg(&g.kap[jj])));
      const T mr = __ldg(&mu[r]);
      T* p1 = tile + (2 * l) * ls + pidx(r);
      T* p2 = tile + (2 * l + 1) * ls + pidx(r);
      const T V1 = *p1, V2 = *p2;
      if (kind == PK_PS) {
        // [[lam, -alpha], [alpha, conj(lam)]] [U1; U2] = [V1; V2], lam = lambda_r + c
        const T lam = mk<R>(mr.x + c, mr.y);
        const R inv = (R)1 / (lam.x * lam.x + lam.y * lam.y + a2);
        *p1 = cscale(cadd(cmul(cconj(lam), V1), cscale(V2, alpha)), inv);
        *p2 = cscale(csub(cmul(lam, V2), cscale(V1, alpha)), inv);
      } else {
        R w;
        if (kind == PK_ABS_PS) {
          const R lx = mr.x + c;
          w = rsqrt_<R>(lx * lx + mr.y * mr.y + a2);
        } else {
          w = (R)1 / (sqrt(mr.x * mr.x + mr.y * mr.y + a2) + c);
        }
        *p1 = cscale(V1, w);
        *p2 = cscale(V2, w);
      }
    }
    __syncthreads();
  }
  const R sc = (R)1 / (R)n;
  for (int e = tid; e < cpb * n; e += nthr) {
    const int l = e % cpb, tt = e / cpb;
    const int col = c0 + l;
    if (col < m) {
      const T w = __ldg(&pr[tt]);
      const T z0 = tile[(2 * l) * ls + pidx(tt)], z1 = tile[(2 * l + 1) * ls + pidx(tt)];
      const long long a = (long long)tt * m + col;
      y[a] = (z0.x * w.x + z0.y * w.y) * sc;        // Re(z conj(w)) / n
      y[mn + a] = (z1.x * w.x + z1.y * w.y) * sc;
    }
  }
}

template <typename R, int Q>
__device__ __forceinline__ void time_body(const Geom& g, int lb, int kind) {
  if (!g.zeta_pi) {
    time_body_general<R, Q>(g, lb, kind);
    return;
  }
  using T = cx<R>;
  R* __restrict__ y = (R*)g.scratch;
  const int n = g.n, m = g.m, N = g.N, cpb = g.time_cpb[sizeof(R) == 4];   // cpb: power of two
  const int ls = padded_len(n);
  const long long mn = g.mn;
  const int c0 = lb * cpb;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = (T*)smem_raw;
  const T* __restrict__ pr = pre<R>(g);
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int csh = __ffs(cpb) - 1;
  {
    const int l = tid & (cpb - 1), ts = nthr >> csh;
    const int col = c0 + l;
    T* dst = tile + l * ls;
    const bool cv = col < m;
    for (int tt = tid >> csh; tt < n; tt += 8 * ts) {
      R a0[8], a1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t2 = tt + u * ts;
        const bool ok = cv && t2 < n;
        const long long a = (long long)t2 * m + col;
        a0[u] = ok ? y[a] : (R)0;
        a1[u] = ok ? y[mn + a] : (R)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t2 = tt + u * ts;
        if (t2 < n) dst[pidx(t2)] = cmul(mk<R>(a0[u], a1[u]), __ldg(&pr[t2]));
      }
    }
  }
  __syncthreads();

  const int P = n / Q;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int lpw = 32 / P;
  const int t = lane % P;
  LaneStages<T, R> stf, sti;
  lane_stages<T, R>(stf, t, P, false);
  lane_stages<T, R>(sti, t, P, true);
  const T* __restrict__ tw = twt<R>(g);
  T twq[Q < 32 ? Q : 1];
  if constexpr (Q < 32) {
#pragma unroll
    for (int k1 = 0; k1 < Q; ++k1) twq[k1] = __ldg(&tw[t * k1]);
  }
  const T* __restrict__ mu = mutab<R>(g);
  const R alpha = (R)g.alpha, a2 = (R)(g.alpha * g.alpha);
  const int half = n / 2;
  const int k2 = bitrev(t, P);
  for (int lbase = warp * lpw; lbase < cpb; lbase += nw * lpw) {
    const int l = lbase + lane / P;
    const bool lv = l < cpb;
    T* line = tile + (lv ? l : 0) * ls;
    const int col = c0 + (lv ? l : 0);
    LineFFT<T, R, Q> f;
    // forward
#pragma unroll
    for (int q = 0; q < Q; ++q) f.x[q] = lv ? line[pidx(t + P * q)] : mk<R>(0, 0);
    __syncwarp();
    f.run(t, P, stf, tw, twq, line, false);
    __syncwarp();
    if (lv) {
#pragma unroll
      for (int j = 0; j < Q; ++j) line[pidx(LineFFT<T, R, Q>::owned(j, t, k2))] = f.value(j);
    }
    __syncwarp();
    // pointwise solve on frequency pairs (r, n-1-r)
    if (lv && col < m) {
      const int j = col / N, i = col - j * N;
      const R c = (R)(g.tau * (__ldg(&g.kap[i]) + __ldg(&g.kap[j])));
      for (int r = t; r < half; r += P) {
        const int rp = n - 1 - r;
        const T mr = __ldg(&mu[r]);
        const T lam = mk<R>(mr.x + c, mr.y);
        const R mod2 = lam.x * lam.x + lam.y * lam.y;
        T* pa = line + pidx(r);
        T* pb = line + pidx(rp);
        if (kind == PK_ABS_PS) {
          const R w = rsqrt_<R>(mod2 + a2);
          *pa = cscale(*pa, w);
          *pb = cscale(*pb, w);
        } else if (kind == PK_PMS) {
          const R sig = sqrt(mr.x * mr.x + mr.y * mr.y + a2);
          const R w = (R)1 / (sig + c);
          *pa = cscale(*pa, w);
          *pb = cscale(*pb, w);
        } else {
          const T Cr = *pa, Cq = cconj(*pb);
          const T F1 = cscale(cadd(Cr, Cq), (R)0.5);
          const T F2 = cmul_mi(cscale(csub(Cr, Cq), (R)0.5));
          const R inv = (R)1 / (mod2 + a2);
          const T U1 = cscale(cadd(cmul(cconj(lam), F1), cscale(F2, alpha)), inv);
          const T U2 = cscale(csub(cmul(lam, F2), cscale(F1, alpha)), inv);
          *pa = cadd(U1, cmul_pi(U2));
          *pb = cadd(cconj(U1), cmul_pi(cconj(U2)));
        }
      }
    }
    __syncwarp();
    // inverse
#pragma unroll
    for (int q = 0; q < Q; ++q) f.x[q] = lv ? line[pidx(t + P * q)] : mk<R>(0, 0);
    __syncwarp();
    f.run(t, P, sti, tw, twq, line, true);
    __syncwarp();
    if (lv) {
#pragma unroll
      for (int j = 0; j < Q; ++j) line[pidx(LineFFT<T, R, Q>::owned(j, t, k2))] = f.value(j);
    }
    __syncwarp();
  }
  __syncthreads();
  const R sc = (R)1 / (R)n;
  {
    const int l = tid & (cpb - 1), ts = nthr >> csh;
    const int col = c0 + l;
    if (col < m) {
      const T* srcs = tile + l * ls;
      for (int tt = tid >> csh; tt < n; tt += ts) {
        const T v = cscale(cmul(srcs[pidx(tt)], cconj(__ldg(&pr[tt]))), sc);
        const long long a = (long long)tt * m + col;
        y[a] = v.x;
        y[mn + a] = v.y;
      }
    }
  }
}

template <typename R, int Q>
__global__ void __launch_bounds__(256, 2) k_time(const Geom* __restrict__ G, const int* __restrict__ off, int count,
                                              Sel sel, int kind) {
  const int inst = find_inst(off, count, blockIdx.x);
  if (sel.skip(inst)) return;
  time_body<R, Q>(G[inst], blockIdx.x - off[inst], kind);
}

template <typename R>
__global__ void __launch_bounds__(256, 2) k_time_any(const Geom* __restrict__ G, const int* __restrict__ off,
                                                  int count, Sel sel, int kind) {
  const int inst = find_inst(off, count, blockIdx.x);
  if (sel.skip(inst)) return;
  const Geom& g = G[inst];
  const int lb = blockIdx.x - off[inst];
  switch (g.time_q) {
    case 1: time_body<R, 1>(g, lb, kind); break;
    case 2: time_body<R, 2>(g, lb, kind); break;
    case 4: time_body<R, 4>(g, lb, kind); break;
    case 8: time_body<R, 8>(g, lb, kind); break;
    case 16: time_body<R, 16>(g, lb, kind); break;
    default: time_body<R, 32>(g, lb, kind); break;
  }
}

// ------------------------------------------------------------------------------------------
// host side: shapes, constant tables, launchers
// ------------------------------------------------------------------------------------------
static int largest_pow2_divisor(int v) { return v & (-v); }

int dst_Q(int M) {
  const int P = std::min(32, largest_pow2_divisor(M));
  return M / P;
}
int time_Q(int n) { return n / std::min(32, n); }
bool q_supported(int Q) {
  return Q == 1 || Q == 2 || Q == 3 || Q == 4 || Q == 6 || Q == 8 || Q == 12 || Q == 16 || Q == 24 || Q == 32;
}
size_t dst_smem_bytes(const Geom& g, int p) {
  const size_t elems = (size_t)std::max(g.dst_lpb[p], g.dst_lpb_j[p]) * padded_len(g.N + 1) +
                       (g.dst_q == 32 ? (size_t)8 * 32 * 33 : 0);   // per-warp transpose scratch
  return elems * (p ? sizeof(float2) : sizeof(double2));
}
int padded_len_host(int len) { return padded_len(len); }
size_t time_smem_bytes(const Geom& g, int p) {
  // general zeta: two complex lines per spatial column
  return (size_t)(g.zeta_pi ? 1 : 2) * g.time_cpb[p] * padded_len(g.n) * (p ? sizeof(float2) : sizeof(double2));
}

cudaError_t pipe_upload_constants();
cudaError_t upload_constants() {
  const cudaError_t e = upload_w96();
  return e != cudaSuccess ? e : pipe_upload_constants();
}

template <typename R, int Q>
static void launch_dst_q(const Batch& B, int axis, int in_slot, int out_slot, int inv, size_t smem) {
  const int p = sizeof(R) == 4;
  static DeviceOnce once;
  once([] {
    cudaFuncSetAttribute(k_dst<double, R, R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_dst<R, R, R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return cudaFuncSetAttribute(k_dst<R, double, R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  const int* off = axis == 0 ? B.off_dst_i[p] : B.off_dst_j[p];
  const int tot = axis == 0 ? B.tot_dst_i[p] : B.tot_dst_j[p];
  if (in_slot >= 0)
    k_dst<double, R, R, Q><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, in_slot, -1, inv);
  else if (out_slot >= 0)
    k_dst<R, double, R, Q><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, -1, out_slot, inv);
  else
    k_dst<R, R, R, Q><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, -1, -1, inv);
}

template <typename R, int Q>
static void launch_time_q(const Batch& B, int kind, size_t smem) {
  const int p = sizeof(R) == 4;
  static DeviceOnce once;
  set_smem_limit(once, k_time<R, Q>, 227 * 1024);
  k_time<R, Q><<<B.tot_time[p], 256, smem, B.stream>>>(B.G, B.off_time[p], B.count, B.sel(), kind);
}

template <typename R>
static cudaError_t dispatch_dst(const Batch& B, int axis, int in_slot, int out_slot, int inv) {
  const int p = sizeof(R) == 4;
  const size_t smem = B.dst_smem[p];
  if (B.dst_q == 0) {   // instances with different line lengths in one launch
    static DeviceOnce once;
    once([] {
      cudaFuncSetAttribute(k_dst_any<double, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      cudaFuncSetAttribute(k_dst_any<R, R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      return cudaFuncSetAttribute(k_dst_any<R, double, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    const int* off = axis == 0 ? B.off_dst_i[p] : B.off_dst_j[p];
    const int tot = axis == 0 ? B.tot_dst_i[p] : B.tot_dst_j[p];
    if (in_slot >= 0)
      k_dst_any<double, R, R><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, in_slot, -1, inv);
    else if (out_slot >= 0)
      k_dst_any<R, double, R><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, -1, out_slot, inv);
    else
      k_dst_any<R, R, R><<<tot, 256, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), axis, -1, -1, inv);
    return cudaGetLastError();
  }
  switch (B.dst_q) {
    case 1: launch_dst_q<R, 1>(B, axis, in_slot, out_slot, inv, smem); break;
    case 2: launch_dst_q<R, 2>(B, axis, in_slot, out_slot, inv, smem); break;
    case 3: launch_dst_q<R, 3>(B, axis, in_slot, out_slot, inv, smem); break;
    case 4: launch_dst_q<R, 4>(B, axis, in_slot, out_slot, inv, smem); break;
    case 6: launch_dst_q<R, 6>(B, axis, in_slot, out_slot, inv, smem); break;
    case 8: launch_dst_q<R, 8>(B, axis, in_slot, out_slot, inv, smem); break;
    case 12: launch_dst_q<R, 12>(B, axis, in_slot, out_slot, inv, smem); break;
    case 16: launch_dst_q<R, 16>(B, axis, in_slot, out_slot, inv, smem); break;
    case 24: launch_dst_q<R, 24>(B, axis, in_slot, out_slot, inv, smem); break;
    case 32: launch_dst_q<R, 32>(B, axis, in_slot, out_slot, inv, smem); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
static cudaError_t dispatch_time(const Batch& B, int kind) {
  const int p = sizeof(R) == 4;
  const size_t smem = B.time_smem[p];
  if (B.time_q == 0) {
    static DeviceOnce once;
    set_smem_limit(once, k_time_any<R>, 227 * 1024);
    k_time_any<R><<<B.tot_time[p], 256, smem, B.stream>>>(B.G, B.off_time[p], B.count, B.sel(), kind);
    return cudaGetLastError();
  }
  switch (B.time_q) {
    case 1: launch_time_q<R, 1>(B, kind, smem); break;
    case 2: launch_time_q<R, 2>(B, kind, smem); break;
    case 4: launch_time_q<R, 4>(B, kind, smem); break;
    case 8: launch_time_q<R, 8>(B, kind, smem); break;
    case 16: launch_time_q<R, 16>(B, kind, smem); break;
    case 32: launch_time_q<R, 32>(B, kind, smem); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t pipe_dst_pass(const Batch& B, int stage, int in_slot, int out_slot);
cudaError_t pipe_time_pass(const Batch& B, int kind);

// FP32 passes take the pipelined kernels (precond_pipe.cu) for the instances whose line shapes
// they cover; a batch that mixes kernel families runs one launch per family present.  `stage` is
// the pass number (1, 2, 4 or 5); the kernels of this file run passes 1 and 5 along x1 and
// passes 2 and 4 along x2.
template <typename R>
static cudaError_t dst_pass(const Batch& B, int stage, int in_slot, int out_slot) {
  const int axis = (stage == 1 || stage == 5) ? 0 : 1;
  const int inv = stage >= 4;          // passes 4 and 5 run the inverse transform (DCT-I pair)
  if (sizeof(R) == 8 || B.pipe_pd == 0) return dispatch_dst<R>(B, axis, in_slot, out_slot, inv);
  if (B.pipe_pd > 0) return pipe_dst_pass(B, stage, in_slot, out_slot);
  Batch F = B;
  F.filt = B.fam_dst;
  for (int b = 0; b < kFamilies; ++b) {
    if (!(B.fam_dst_set >> b & 1)) continue;
    F.filt_want = fam_code(b);
    F.pipe_pd = F.filt_want;
    const cudaError_t e = b ? pipe_dst_pass(F, stage, in_slot, out_slot) : dispatch_dst<R>(F, axis, in_slot, out_slot, inv);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
template <typename R>
static cudaError_t time_pass(const Batch& B, int kind) {
  if (sizeof(R) == 8 || B.pipe_pt == 0) return dispatch_time<R>(B, kind);
  if (B.pipe_pt > 0) return pipe_time_pass(B, kind);
  Batch F = B;
  F.filt = B.fam_time;
  for (int b = 0; b < kFamilies; ++b) {
    if (!(B.fam_time_set >> b & 1)) continue;
    F.filt_want = fam_code(b);
    F.pipe_pt = F.filt_want;
    const cudaError_t e = b ? pipe_time_pass(F, kind) : dispatch_time<R>(F, kind);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
static cudaError_t precond_passes(const Batch& B, int kind, int in_slot, int out_slot) {
  cudaError_t e;
  if ((e = dst_pass<R>(B, 1, in_slot, -1)) != cudaSuccess) return e;
  if ((e = dst_pass<R>(B, 2, -1, -1)) != cudaSuccess) return e;
  if ((e = time_pass<R>(B, kind)) != cudaSuccess) return e;
  if ((e = dst_pass<R>(B, 4, -1, -1)) != cudaSuccess) return e;
  return dst_pass<R>(B, 5, -1, out_slot);
}

int precond_launch_count(bool var_a, int kind) { return var_a ? mg_launch_count(kind) : 5; }

// ------------------------------------------------------------------------------------------
// Finite elements (M != I, Sec. 1): the spatial operator K~ = M^{-1/2} K M^{-1/2} is diagonal in the
// sine basis, so products with it, and with M^{1/2} and M^{-1/2}, run as FP64 2D DST-I, a per-mode
// step, and the inverse DST-I (the DST-I is its own inverse).  The per-mode step works in place on
// the problem's FP64 scratch, which the two DST passes leave in the vector layout with mode
// (p, q) at the position of node (p, q).
// ------------------------------------------------------------------------------------------
enum { FEM_MASS_SQRT = 0, FEM_MASS_ISQRT = 1, FEM_PRODUCT = 2 };

// One thread per mode col = (p, q), both halves, all time steps.
//   FEM_MASS_SQRT / FEM_MASS_ISQRT: scale by (mu_p mu_q)^{+1/2} / ^{-1/2}.
//   FEM_PRODUCT: the all-at-once product (Eq. matrix_A or matrix_A_hat) with K~ diagonal:
//     T x1 = B_n x1 + tau kappa x1, B_n = B1 B2^{-1}: z_t = (x1_t - (1-theta) z_{t-1}) / theta, z_t - z_{t-1};
//     T^T x2 = B1^T B2^{-T} x2 + tau kappa x2: u_t = (x2_t - (1-theta) u_{t+1}) / theta, u_t - u_{t+1}.
//   The backward sweep parks u in the first half of `tmp` (a vector the caller overwrites later);
//   the forward sweep then reads x1_t, x2_t and writes both outputs at t, after which nothing reads t.
__global__ void __launch_bounds__(256) k_fem_modal(const Geom* __restrict__ G, const Slots* __restrict__ S, int mode,
                                                   int op, int tmp_slot) {
  const Geom& g = G[0];
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.m) return;
  const int N = g.N, n = g.n, m = g.m;
  const long long mn = g.mn;
  const int q = col / N, p = col - q * N;
  double* __restrict__ w = (double*)g.scratch;
  if (mode != FEM_PRODUCT) {
    const double mu = __ldg(&g.mass[p]) * __ldg(&g.mass[q]);
    const double sc = mode == FEM_MASS_SQRT ? sqrt(mu) : 1.0 / sqrt(mu);
    for (int t = 0; t < n; ++t) {
      const long long a = (long long)t * m + col;
      w[a] *= sc;
      w[mn + a] *= sc;
    }
    return;
  }
  const double tk = g.tau * (__ldg(&g.kap[p]) + __ldg(&g.kap[q]));
  const double th = g.theta, om = 1.0 - th, ith = 1.0 / th, alpha = g.alpha;
  double* __restrict__ ubuf = S[0].v[tmp_slot];
  const double* __restrict__ x1 = w;
  const double* __restrict__ x2 = w + mn;
  double unext = 0.0;
  for (int t = n - 1; t >= 0; --t) {
    const long long a = (long long)t * m + col;
    const double u = fma(-om, unext, x2[a]) * ith;
    ubuf[a] = u;
    unext = u;
  }
  const long long offT = op == PCB_OP_A ? mn : 0, offTT = op == PCB_OP_A ? 0 : mn;
  double zprev = 0.0;
  for (int t = 0; t < n; ++t) {
    const long long a = (long long)t * m + col;
    const double x1c = x1[a], x2c = x2[a];
    const double z = fma(-om, zprev, x1c) * ith;
    const double un = t + 1 < n ? ubuf[a + m] : 0.0;
    double oT = (z - zprev) + tk * x1c;
    oT = fma(-alpha, x2c, oT);
    double oTT = (ubuf[a] - un) + tk * x2c;
    oTT = fma(alpha, x1c, oTT);
    w[offT + a] = oT;
    w[offTT + a] = oTT;
    zprev = z;
  }
}

// y = Op x through the sine basis; in_slot, out_slot: vector slots (they may coincide for the mass
// factors; the product needs distinct ones, out_slot serving as the sweep's temporary).
cudaError_t launch_fem_spatial(const Batch& B, int mode, int op, int in_slot, int out_slot) {
  cudaError_t e;
  if ((e = dst_pass<double>(B, 1, in_slot, -1)) != cudaSuccess) return e;
  if ((e = dst_pass<double>(B, 2, -1, -1)) != cudaSuccess) return e;
  k_fem_modal<<<(B.fem_m + 255) / 256, 256, 0, B.stream>>>(B.G, B.S, mode, op, out_slot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = dst_pass<double>(B, 4, -1, -1)) != cudaSuccess) return e;
  return dst_pass<double>(B, 5, -1, out_slot);
}

// B.dst_q / B.time_q = 0 selects the shared-launch kernels for instances of different sizes.
cudaError_t launch_precond_fast(const Batch& B, int kind, int prec, int in_slot, int out_slot) {
  return prec == PCB_MIXED ? precond_passes<float>(B, kind, in_slot, out_slot)
                           : precond_passes<double>(B, kind, in_slot, out_slot);
}

}  // namespace pcb
