// Pipelined FP32 preconditioner passes for power-of-two line lengths (paper Sec. 3.5).
//
// The same five passes as precond.cu: DST-I along x1, DST-I along x2, time DFT + pointwise
// solve + inverse time DFT, DST-I along x2, DST-I along x1 (for Neumann problems the DCT-I pair
// of the even extension, template flag EV).  They are organised for this GPU as follows.
//   * A line of length M = 32 P (2 <= P <= 32) is transformed by P lanes holding 32 values each,
//     as a two-stage FFT.  With s = t + P q and k = k1 + 32 k2,
//         X[k1 + 32 k2] = sum_t W_P^{t k2} W_M^{t k1} sum_q x[t + P q] W_32^{q k1},
//     that is a 32-point register DFT per lane, the twiddle W_M^{t k1}, an exchange through a
//     per-warp shared-memory block (XOR-swizzled, free of bank conflicts) and 32/P register DFTs
//     of size P.  Lane t starts with x[t + P q] and ends with X[u + P j] (u = t).  Both orders
//     are cyclic with stride P, so contiguous lines load and store coalesced, with no bit
//     reversal.  The inverse runs the same steps in reverse order.
//   * Every DST pass reads contiguous lines.  Passes 1 and 4 write their result transposed
//     (the two spatial axes swap), so the x2 lines of pass 2 and the x1 lines of pass 5 are
//     contiguous too.  Each warp copies its next line with 16-byte cp.async copies while it
//     transforms the current one.
//   * The FP32 scratch holds two buffers whose rows are padded to 64-byte boundaries (Geom::lr,
//     Geom::mp): x -> buffer 0 (transposed) -> in place -> time pass in place -> buffer 1
//     (transposed back) -> y.
//   * The time pass stages tiles of spatial columns with cp.async (one line per warp for n = 512).
// Two 256-thread blocks run per SM (128 registers, at most about 110 KB of shared memory).  An
// instance takes these kernels for all of its DST passes or for none; see pipe_dst_p.
#include <algorithm>

#include "fft_reg.cuh"

namespace pcb {

namespace {

enum { PK_ABS_PS = 1, PK_PS = 2, PK_PMS = 3 };
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kScrWarp = 1056;        // complex elements of transpose scratch per warp

// ------------------------------------------------------------------------------------------
// asynchronous global -> shared copies
// ------------------------------------------------------------------------------------------
template <int BYTES>
__device__ __forceinline__ void cp_async(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? BYTES : 0;          // 0 source bytes: the destination is zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gsrc), "n"(BYTES), "r"(n)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
  float2 c;
  c.x = a.x * b.x + a.y * b.y;
  c.y = a.y * b.x - a.x * b.y;
  return c;
}

// FP64 <-> FP32 conversions with integer operations.  The conversion instructions run on the FP64
// pipe, which is narrow on this GPU and became the bottleneck of the passes that read or write
// the FP64 vectors.  IEEE-754 binary64 -> binary32, round to nearest even: for results in the
// normal FP32 range the rounded value is the top 31 bits of (exponent - 896, mantissa >> 29)
// plus one when the dropped 29 bits exceed half, or equal half and the kept value is odd (a
// carry into the exponent gives the right next binade, or infinity).  Zeros keep their sign;
// the rare remaining cases (FP32 subnormals, overflow, infinities, NaN) use the instruction.
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ah = hi & 0x7fffffffu, e = ah >> 20;
  if (e - 897u <= 253u) {
    const unsigned m = (ah << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    const unsigned rnd = (unsigned)(rem > 0x10000000u) | ((unsigned)(rem == 0x10000000u) & m & 1u);
    return __uint_as_float(((m - (896u << 23)) + rnd) | (hi & 0x80000000u));
  }
  if ((ah | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return __double2float_rn(x);
}
// binary32 -> binary64 (exact): exponent rebiased by 896, mantissa moved up by 29 bits
__device__ __forceinline__ double f2d(float f) {
  const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xffu;
  if (e - 1u < 254u) {
    const unsigned hi = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(b << 29));
  }
  if ((b & 0x7fffffffu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)f;
}
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return d2f(v); }
// The gather of pass 1 converts every kF2FEvery-th register of a line with the conversion
// instruction and the rest with integer operations: both round to nearest even, and the mix
// shares the work between the FP64 pipe and the integer pipe.
constexpr int kF2FEvery = 2;
__device__ __forceinline__ float to_f32_at(float v, int) { return v; }
__device__ __forceinline__ float to_f32_at(double v, int q) {
  return (kF2FEvery > 0 && q % kF2FEvery == kF2FEvery - 1) ? __double2float_rn(v) : d2f(v);
}
template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ double from_f32<double>(float v) { return f2d(v); }
// pass 5's FP64 results: every kF2DEvery-th register through the conversion instruction
constexpr int kF2DEvery = 2;
template <typename T> __device__ __forceinline__ T from_f32_at(float v, int j) {
  if constexpr (sizeof(T) == 8) {
    if (kF2DEvery > 0 && j % kF2DEvery == kF2DEvery - 1) return (double)v;
  }
  return from_f32<T>(v);
}

// ------------------------------------------------------------------------------------------
// two-stage line FFT, M = 32 P
// ------------------------------------------------------------------------------------------
template <int P>
struct Two {
  static constexpr int A = 32 / P;    // stage-2 DFTs per lane
  // register that holds X[u + P j] after fwd()
  __device__ static constexpr int outreg(int j) { return (j % A) * P + pos<P>(j / A); }
  // complex offset of (k1, t) in a group's exchange block: row k1, column t XOR-swizzled by k1
  __device__ static constexpr int sidx(int k1, int t) { return k1 * P + (t ^ (k1 & (P - 1))); }
};

// forward: x[q] = v[t + P q] on entry; X[t + P j] in x[Two<P>::outreg(j)] on exit.
// tw2[k1 P + t] = W_M^{t k1}.
template <int P>
__device__ __forceinline__ void fwd2(float2* x, int t, float2* __restrict__ scr, const float2* __restrict__ tw2) {
  reg_dft<float2, float, 32>(x, false);
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) {
    float2 v = x[pos<32>(k1)];
    if (k1) v = cmul(v, tw2[k1 * P + t]);
    scr[Two<P>::sidx(k1, t)] = v;
  }
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 32 / P; ++a)
#pragma unroll
    for (int tt = 0; tt < P; ++tt) x[a * P + tt] = scr[(t + P * a) * P + (tt ^ t)];
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 32 / P; ++a) reg_dft<float2, float, P>(x + a * P, false);
}

// inverse (unnormalised): X[u + P j] in x[Two<P>::outreg(j)] on entry; M v[u + P q] in
// x[pos<32>(q)] on exit.  tw3[(a P + t) P + u] = W_M^{t (u + P a)}.
template <int P>
__device__ __forceinline__ void inv2(float2* x, int u, float2* __restrict__ scr, const float2* __restrict__ tw3) {
#pragma unroll
  for (int a = 0; a < 32 / P; ++a) {
    float2 z[P];
#pragma unroll
    for (int k2 = 0; k2 < P; ++k2) z[k2] = x[a * P + pos<P>(k2)];
    reg_dft<float2, float, P>(z, true);
#pragma unroll
    for (int tt = 0; tt < P; ++tt) {
      float2 v = z[pos<P>(tt)];
      if (tt) v = cmulc(v, tw3[(a * P + tt) * P + u]);
      scr[(u + P * a) * P + (tt ^ u)] = v;
    }
  }
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) x[k1] = scr[Two<P>::sidx(k1, u)];
  __syncwarp();
  reg_dft<float2, float, 32>(x, true);
}

// twiddle tables of one line length from W_M^k (k < M) in global memory
template <int P>
__device__ __forceinline__ void fill_twiddles(float2* tw2, float2* tw3, const float2* __restrict__ w) {
  constexpr int M = 32 * P;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int t2 = k % P, k1 = k / P;
    tw2[k] = __ldg(&w[t2 * k1]);
    if (tw3) {
      const int u = k % P, tt = (k / P) % P, a = k / (P * P);
      tw3[k] = __ldg(&w[tt * (u + P * a)]);
    }
  }
}

// tile line pitch (complex elements): >= len, chosen so that the strided tile loads of the
// x2-line and time passes spread over the shared-memory banks
template <int P>
__host__ __device__ constexpr int pitch_for(int len) {
  const int r = P >= 16 ? P / 8 : 1;   // residue mod 16
  return len + ((r - len % 16) + 16) % 16;
}

// an instance of this launch's family with work: the source of the tables that depend on the
// line length only
__device__ __forceinline__ int table_inst(const int* __restrict__ off, int count, Sel sel) {
  if (!sel.fam) return find_inst(off, count, 0);
  for (int k = 0; k < count; ++k)
    if (__ldg(sel.fam + k) == sel.want && __ldg(off + k + 1) > __ldg(off + k)) return k;
  return 0;
}

// forward transform of an odd line (z_{M-s} = -z_s): as fwd2, but the exchange keeps only the
// columns t <= P/2.  For t = P - t' (1 <= t' < P/2) the stage-1 outputs are redundant:
//     V[P-t'][k1] = -W_P^{-t'} V[t'][32-k1]  (k1 != 0),   V[P-t'][0] = -V[t'][0],
// with V[t][k1] = W_M^{t k1} sum_q z_{t+Pq} W_32^{q k1}, so readers rebuild them from the stored
// half (shared memory per group: 32 rows x (P/2 + 1) columns).  wP[k] = W_P^k.  EV: an even line
// (z_{M-s} = z_s, the DCT-I extension) has the same relation with the opposite sign.
template <int P, bool EV = false>
__device__ __forceinline__ void fwd_odd(float2* x, int t, float2* __restrict__ scr, const float2* __restrict__ tw2,
                                        const float2* __restrict__ wP) {
  constexpr int CW = P / 2 + 1;
  reg_dft<float2, float, 32>(x, false);
  if (t <= P / 2) {
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) {
      float2 v = x[pos<32>(k1)];
      if (k1) v = cmul(v, tw2[k1 * P + t]);
      scr[k1 * CW + t] = v;
    }
  }
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 32 / P; ++a) {
    const int k1 = t + P * a;
    const int k1m = (32 - k1) & 31;
    const bool z0 = k1 == 0;
#pragma unroll
    for (int tt = 0; tt < P; ++tt) {
      if (tt <= P / 2) {
        x[a * P + tt] = scr[k1 * CW + tt];
      } else {
        const float2 sv = scr[k1m * CW + (P - tt)];
        const float2 w = wP[tt];
        const float sgn = EV ? 1.f : -1.f;
        float2 mlt;
        mlt.x = z0 ? sgn : sgn * w.x;
        mlt.y = z0 ? 0.f : sgn * w.y;
        x[a * P + tt] = cmul(sv, mlt);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int a = 0; a < 32 / P; ++a) reg_dft<float2, float, P>(x + a * P, false);
}

template <int P>
__host__ __device__ constexpr int odd_scratch_per_warp() { return (32 / P) * 32 * (P / 2 + 1); }

// DST-I tables: tw2 (M entries, see fwd2) and wP[k] = W_P^k = W_M^{32 k}
template <int P>
__device__ __forceinline__ void fill_dst_tables(float2* tw2, float2* wP, const float2* __restrict__ w) {
  fill_twiddles<P>(tw2, nullptr, w);
  for (int k = threadIdx.x; k < P; k += blockDim.x) wP[k] = __ldg(&w[32 * k]);
}

// ------------------------------------------------------------------------------------------
// DST-I along x1 (contiguous lines of N = 16 P - 1 values).  Warps work independently, one line
// at a time: the line's two halves are fetched with 16-byte cp.async copies into the warp's
// shared-memory slot (the 16-byte aligned span that covers the line), gathered into registers,
// and the copy of the warp's next line is issued before the line is transformed.  The result is
// stored straight from registers (lane u holds S_p, p = u + P j: consecutive lanes, consecutive
// addresses).  Tiles of LPB = 256 / P lines give the block offsets.
// in_sel / out_sel >= 0: FP64 vector slot; -1 / -2: FP32 scratch buffer 0 / 1.
// ------------------------------------------------------------------------------------------
// Layout of the vector a pass reads or writes: slot sel >= 0 of the instance (FP64, rows of N,
// slices of m, halves of mn values) or FP32 scratch buffer -1 - sel (rows of lr, slices of mp,
// halves of n mp values).  Element (half h, time t, row r, index i) sits at
// base + h hs + t ts + r rs + i.
struct View {
  void* base;
  long long hs, ts;
  int rs;
};
__device__ __forceinline__ View view_of(const Geom& g, const Slots& s, int sel) {
  View v;
  if (sel >= 0) {
    v.base = s.v[sel]; v.hs = g.mn; v.ts = g.m; v.rs = g.N;
  } else {
    v.hs = (long long)g.n * g.mp; v.ts = g.mp; v.rs = g.lr;
    v.base = (float*)g.scratch + (sel == -1 ? 0 : 2 * v.hs);
  }
  return v;
}

// values per spatial line of the pipelined passes: DST-I lines hold N = L - 1 interior values, the
// DCT-I lines of the Neumann grid N = L + 1 nodes (L = 16 P, the line FFT has M = 2 L points)
template <int P, bool EV>
__host__ __device__ constexpr int line_values() { return EV ? 16 * P + 1 : 16 * P - 1; }

template <typename TIn>
__host__ __device__ constexpr int row_slot_elems(int N) {   // per half: N values + both alignment tails
  return ((N + 32 / (int)sizeof(TIn) + 16 / (int)sizeof(TIn) - 1) / (16 / (int)sizeof(TIn))) * (16 / (int)sizeof(TIn));
}

// EV: the DCT-I pair of the Neumann route instead (lines of N = L + 1 nodes, even extension);
// inv = 1 selects the inverse of the pair (end values scaled by sqrt 2 on input), inv = 0 the
// forward one (end modes scaled by sqrt 1/2 on output).
template <typename TIn, typename TOut, int P, bool EV>
__global__ void __launch_bounds__(kThreads, 2)
    k_dst_rows(const Geom* __restrict__ G, const Slots* __restrict__ S, const int* __restrict__ off, int count,
               Sel sel, int in_sel, int out_sel, int tot, int inv) {
  constexpr int M = 32 * P, L = 16 * P, N = line_values<P, EV>(), LPB = kThreads / P;
  constexpr int EPC = 16 / (int)sizeof(TIn);              // elements per 16-byte chunk
  constexpr int SLOT = row_slot_elems<TIn>(N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* wP = tw2 + M;
  float2* scr_all = wP + P;
  TIn* slots = (TIn*)(scr_all + kWarps * odd_scratch_per_warp<P>());
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  fill_dst_tables<P>(tw2, wP, G[table_inst(off, count, sel)].twd_f);
  __syncthreads();
  float2* scr = scr_all + warp * odd_scratch_per_warp<P>() + (lane / P) * 32 * (P / 2 + 1);
  TIn* slot = slots + (size_t)warp * (32 / P) * 2 * SLOT;   // (32/P) lines x 2 halves
  const int t = lane % P, grp = lane / P;
  const float sc = __frsqrt_rn((float)(2 * L));     // DST-I normalisation 0.5 sqrt(2/L)
  const long long nvt = (long long)tot * kWarps;

  // the warp's lines of work item vt (tile vt / 8, warp slot vt % 8): group k has line line0 + k
  struct Item { int inst; long long line0; int nl; };    // nl: valid lines (0: nothing to do)
  auto decode = [&](long long vt) {
    Item it{0, 0, 0};
    if (vt >= nvt) return it;
    const int tile = (int)(vt / kWarps), w = (int)(vt % kWarps);
    it.inst = find_inst(off, count, tile);
    if (sel.skip(it.inst)) return it;
    const long long nlines = (long long)G[it.inst].n * N;
    it.line0 = (long long)(tile - off[it.inst]) * LPB + w * (32 / P);
    it.nl = (int)min((long long)(32 / P), max(0LL, nlines - it.line0));
    return it;
  };
  // line l = t N + r of the item's instance: offset t ts + r rs in a view
  auto line_off = [&](const View& v, long long l) { return (l / N) * v.ts + (l % N) * v.rs; };
  // copy the 16-byte aligned spans covering the item's lines (both halves) into the slot
  auto issue = [&](const Item& it) {
    if (it.nl > 0) {
      const View v = view_of(G[it.inst], S[it.inst], in_sel);
      for (int k = 0; k < it.nl; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const TIn* base = (const TIn*)v.base + h * v.hs + line_off(v, it.line0 + k);
          const char* a0 = (const char*)((uintptr_t)base & ~(uintptr_t)15);
          const char* a1 = (const char*)(((uintptr_t)(base + N) + 15) & ~(uintptr_t)15);
          const int nch = (int)((a1 - a0) >> 4);
          TIn* d = slot + (k * 2 + h) * SLOT;
          for (int c = lane; c < nch; c += 32) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(d + c * EPC);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(a0 + 16 * c) : "memory");
          }
        }
      }
    }
    cp_commit();
  };

  long long vt = (long long)blockIdx.x * kWarps + warp;
  const long long stride = (long long)gridDim.x * kWarps;
  Item cur = decode(vt);
  issue(cur);
  for (; vt < nvt; vt += stride) {
    const Item nxt = decode(vt + stride);
    cp_wait<0>();
    __syncwarp();
    const bool lv = grp < cur.nl;
    float2 x[32];
    if (cur.nl > 0) {
      const View v = view_of(G[cur.inst], S[cur.inst], in_sel);
      const TIn* in = (const TIn*)v.base + line_off(v, cur.line0 + (lv ? grp : 0));
      const int o0 = (int)(((uintptr_t)in & 15) / sizeof(TIn));
      const int o1 = (int)(((uintptr_t)(in + v.hs) & 15) / sizeof(TIn));
      const TIn* s0 = slot + (lv ? grp : 0) * 2 * SLOT + o0;
      const TIn* s1 = slot + ((lv ? grp : 0) * 2 + 1) * SLOT + o1;
      // gather the odd extension: z_s = x_{s-1} (1 <= s <= N), -x_{M-s-1} (L < s < M), 0 else;
      // EV: the even one, z_s = x_s (s <= L), x_{M-s} (L < s < M)
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int s = t + P * q;
        if constexpr (EV) {
          const int idx = q < 16 ? s : M - s;
          float2 v = make_float2(to_f32(s0[idx]), to_f32(s1[idx]));
          if (!lv) v = make_float2(0.f, 0.f);
          if (inv && (s == 0 || s == L)) v = cscale(v, 1.41421356237309515f);
          x[q] = v;
        } else {
          const bool ok = lv && (q < 16 ? s > 0 : s > L);
          const int idx = q < 16 ? (s > 0 ? s - 1 : 0) : (s > L ? M - s - 1 : 0);
          float2 v = make_float2(to_f32(s0[idx]), to_f32(s1[idx]));
          if (!ok) v = make_float2(0.f, 0.f);
          if (q >= 16) { v.x = -v.x; v.y = -v.y; }
          x[q] = v;
        }
      }
    }
    __syncwarp();
    issue(nxt);                          // the next line's copy overlaps this line's transform
    if (cur.nl > 0) {
      fwd_odd<P, EV>(x, t, scr, tw2, wP);
      if (lv) {
        const View v = view_of(G[cur.inst], S[cur.inst], out_sel);
        TOut* __restrict__ d = (TOut*)v.base + line_off(v, cur.line0 + grp);
        if constexpr (EV) {
          // modes k = t + P j, j <= 16 (k = L only at lane 0); the real transform of each half
          // stays in its own component
#pragma unroll
          for (int j = 0; j <= 16; ++j) {
            const int k = t + P * j;
            if (k <= L) {
              const float2 Y = x[Two<P>::outreg(j)];
              const float f = (!inv && (k == 0 || k == L)) ? sc * 0.707106781186547524f : sc;
              d[k] = from_f32_at<TOut>(Y.x * f, j);
              d[v.hs + k] = from_f32_at<TOut>(Y.y * f, j);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int p = t + P * j;
            const float2 Y = x[Two<P>::outreg(j)];
            if (p >= 1) {
              d[p - 1] = from_f32_at<TOut>(-Y.y * sc, j);
              d[v.hs + p - 1] = from_f32_at<TOut>(Y.x * sc, j);
            }
          }
        }
      }
    }
    cur = nxt;
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// DST-I of contiguous lines with a transposed result.  Tile (t0, r0) is the lines r0 .. r0+LPB-1
// of time step t0 (each N contiguous values of the input buffer); the result of line r at index
// p goes to out[t0 m + p N + r], i.e. the two spatial axes swap.  Passes 1 and 4 use it, so
// that passes 2 and 5 find their lines contiguous as well:
//   pass 1: x (x1 lines) -> buffer 0 with x2 lines contiguous; pass 2 transforms buffer 0 in place;
//   pass 4: buffer 0 -> buffer 1 with x1 lines contiguous again; pass 5: buffer 1 -> y.
// Each warp copies its next lines with cp.async while it transforms the current ones; a warp
// parks its results in its own exchange block, and the block writes the tile out as LPB-wide
// row segments.
// ------------------------------------------------------------------------------------------
template <int P>
__host__ __device__ constexpr int rowsT_region() {   // complex elements per warp: exchange / parked results
  return ((odd_scratch_per_warp<P>() + 11) / 16) * 16 + 4;
}

// MODE 1 (pass 2 when the time lines are 512 long): tile (r, t0) is the lines (t0 + l, r) of the
// rows r of LPB consecutive time steps, and the result goes to the time-major layout of scratch
// buffer 1, value (half h, spatial point r N + p, time t) at h n m + (r N + p) n + t, so that the
// time pass reads contiguous time lines.
template <typename TIn, int P, int MODE, bool EV>
__global__ void __launch_bounds__(kThreads, 2)
    k_dst_rowsT(const Geom* __restrict__ G, const Slots* __restrict__ S, const int* __restrict__ off, int count,
                Sel sel, int in_sel, int out_sel, int tot, int inv) {
  constexpr int M = 32 * P, L = 16 * P, N = line_values<P, EV>(), LPB = kThreads / P, A = 32 / P;
  constexpr int NBT = (N + LPB - 1) / LPB;       // tiles per time step
  constexpr int EPC = 16 / (int)sizeof(TIn);
  constexpr int SLOT = row_slot_elems<TIn>(N);
  constexpr int RS = rowsT_region<P>();
  static_assert(A * N <= RS, "parked results must fit the exchange block");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* wP = tw2 + M;
  float2* regions = wP + P;
  TIn* slots = (TIn*)(regions + kWarps * RS);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  fill_dst_tables<P>(tw2, wP, G[table_inst(off, count, sel)].twd_f);
  float2* region = regions + warp * RS;
  float2* scr = region + (lane / P) * 32 * (P / 2 + 1);
  TIn* slot = slots + (size_t)warp * A * 2 * SLOT;
  const int t = lane % P, grp = lane / P;
  const float sc = __frsqrt_rn((float)(2 * L));

  struct Item { int inst; int t0, r0; int nl; };   // nl: valid lines of this warp (0: none)
  auto decode = [&](int tile) {
    Item it{0, 0, 0, 0};
    if (tile >= tot) return it;
    it.inst = find_inst(off, count, tile);
    if (sel.skip(it.inst)) return it;
    const int lt = tile - off[it.inst];
    if (MODE == 0) {
      it.t0 = lt / NBT;
      it.r0 = (lt - it.t0 * NBT) * LPB;
      it.nl = max(0, min(A, N - (it.r0 + warp * A)));
    } else {
      const int ntt = G[it.inst].n / LPB;        // tiles per row
      it.r0 = lt / ntt;
      it.t0 = (lt - it.r0 * ntt) * LPB;
      it.nl = max(0, min(A, G[it.inst].n - (it.t0 + warp * A)));
    }
    return it;
  };
  auto line_ptr = [&](const Item& it, int k, int h) {
    const View v = view_of(G[it.inst], S[it.inst], in_sel);
    if (MODE == 0)
      return (const TIn*)v.base + h * v.hs + it.t0 * v.ts + (long long)(it.r0 + warp * A + k) * v.rs;
    return (const TIn*)v.base + h * v.hs + (it.t0 + warp * A + k) * v.ts + (long long)it.r0 * v.rs;
  };
  // The 16-byte aligned span of a line is copied in 16-byte pieces.  Where that span would
  // leave the vector (a caller's buffer that is not 16-byte aligned), the line is copied value by
  // value to the same slot positions instead.
  auto issue = [&](const Item& it) {
    if (it.nl > 0) {
      const View v = view_of(G[it.inst], S[it.inst], in_sel);
      const char* lo = (const char*)v.base;
      const char* hi = lo + 2 * v.hs * (long long)sizeof(TIn);
      for (int k = 0; k < it.nl; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const TIn* base = line_ptr(it, k, h);
          const char* a0 = (const char*)((uintptr_t)base & ~(uintptr_t)15);
          const char* a1 = (const char*)(((uintptr_t)(base + N) + 15) & ~(uintptr_t)15);
          TIn* d = slot + (k * 2 + h) * SLOT;
          if (a0 >= lo && a1 <= hi) {
            const int nch = (int)((a1 - a0) >> 4);
            for (int c = lane; c < nch; c += 32) {
              const unsigned sa = (unsigned)__cvta_generic_to_shared(d + c * EPC);
              asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(a0 + 16 * c) : "memory");
            }
          } else {
            TIn* de = d + (((uintptr_t)base & 15) / sizeof(TIn));
            for (int e = lane; e < N; e += 32) cp_async<sizeof(TIn)>(de + e, base + e, true);
          }
        }
      }
    }
    cp_commit();
  };

  Item cur = decode(blockIdx.x);
  issue(cur);
  for (int tile = blockIdx.x; tile < tot; tile += gridDim.x) {
    const Item nxt = decode(tile + gridDim.x);
    const int inst = find_inst(off, count, tile);
    const bool on = !sel.skip(inst);
    cp_wait<0>();
    __syncthreads();                               // tables (first tile) and all slots ready
    const bool lv = grp < cur.nl;
    float2 x[32];
    if (on) {
      const TIn* s0 = slot + (lv ? grp : 0) * 2 * SLOT;
      const TIn* s1 = s0 + SLOT;
      if (lv) {
        s0 += (int)(((uintptr_t)line_ptr(cur, grp, 0) & 15) / sizeof(TIn));
        s1 += (int)(((uintptr_t)line_ptr(cur, grp, 1) & 15) / sizeof(TIn));
      }
      // FP64 input: each value is read and converted once; the mirrored half (q >= 16) comes from
      // the lane holding it: -x_{M-s-1} with s = t + P q is lane P - t's value at q' = 31 - q
      // (lane 0: its own value at 32 - q).  EV (even extension, x_{M-s} at s > L): the same lanes
      // and registers without the sign; lane 0 at q = 16 holds x_L, read from the slot.
      constexpr bool kShuffleMirror = sizeof(TIn) == 8;
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int s = t + P * q;
        if (kShuffleMirror && q >= 16) {
          const float2 a = x[31 - q];
          float2 v;
          v.x = __shfl_sync(0xffffffffu, a.x, (P - t) & (P - 1), P);
          v.y = __shfl_sync(0xffffffffu, a.y, (P - t) & (P - 1), P);
          if constexpr (EV) {
            if (t == 0) {
              v = q > 16 ? x[32 - q] : make_float2(to_f32(s0[L]), to_f32(s1[L]));
              if (q == 16 && !lv) v = make_float2(0.f, 0.f);
              if (q == 16 && inv) v = cscale(v, 1.41421356237309515f);
            }
            x[q] = v;
          } else {
            if (t == 0) v = q > 16 ? x[32 - q] : make_float2(0.f, 0.f);
            x[q] = make_float2(-v.x, -v.y);
          }
          continue;
        }
        if constexpr (EV) {
          const int idx = q < 16 ? s : M - s;
          float2 v = make_float2(to_f32_at(s0[idx], q), to_f32_at(s1[idx], q));
          if (!lv) v = make_float2(0.f, 0.f);
          if (inv && (s == 0 || s == L)) v = cscale(v, 1.41421356237309515f);
          x[q] = v;
        } else {
          const bool ok = lv && (q < 16 ? s > 0 : s > L);
          const int idx = q < 16 ? (s > 0 ? s - 1 : 0) : (s > L ? M - s - 1 : 0);
          float2 v = make_float2(to_f32_at(s0[idx], q), to_f32_at(s1[idx], q));
          if (!ok) v = make_float2(0.f, 0.f);
          if (q >= 16) { v.x = -v.x; v.y = -v.y; }
          x[q] = v;
        }
      }
    }
    __syncwarp();
    issue(nxt);
    if (on) {
      fwd_odd<P, EV>(x, t, scr, tw2, wP);
      __syncwarp();                                // exchange reads done: park the results
      if constexpr (EV) {
#pragma unroll
        for (int j = 0; j <= 16; ++j) {
          const int k = t + P * j;
          if (k <= L) {
            const float2 Y = x[Two<P>::outreg(j)];
            const float f = (!inv && (k == 0 || k == L)) ? sc * 0.707106781186547524f : sc;
            region[grp * N + k] = cscale(Y, f);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int p = t + P * j;
          const float2 Y = x[Two<P>::outreg(j)];
          if (p >= 1) region[grp * N + p - 1] = make_float2(-Y.y * sc, Y.x * sc);
        }
      }
    }
    __syncthreads();
    if (on && MODE == 0) {
      const Geom& g = G[inst];
      const int lt = tile - off[inst];
      const int t0 = lt / NBT, r0 = (lt - t0 * NBT) * LPB;
      const int l = tid % LPB;
      if (r0 + l < N) {
        const View ov = view_of(g, S[inst], out_sel);
        float* d = (float*)ov.base + t0 * ov.ts + r0 + l;
        const float2* src = regions + (l / A) * RS + (l % A) * N;
        for (int p = tid / LPB; p < N; p += kThreads / LPB) {
          const float2 v = src[p];
          d[(long long)p * ov.rs] = v.x;
          d[ov.hs + (long long)p * ov.rs] = v.y;
        }
      }
    } else if (on) {
      const Geom& g = G[inst];
      const int l = tid % LPB;
      if (cur.t0 + l < g.n) {
        const long long hs = (long long)g.n * g.m;
        float* d = (float*)g.scratch + 2LL * g.n * g.mp + (long long)cur.r0 * N * g.n + cur.t0 + l;
        const float2* src = regions + (l / A) * RS + (l % A) * N;
        for (int p = tid / LPB; p < N; p += kThreads / LPB) {
          const float2 v = src[p];
          d[(long long)p * g.n] = v.x;
          d[hs + (long long)p * g.n] = v.y;
        }
      }
    }
    cur = nxt;
  }
  cp_wait<0>();
}

// Pointwise solve at one F-slot r (Sec. 3.5): Cr = coefficient at r, Cq = conj(coefficient at n-1-r),
// mr = lambda(S_n) at r, c = tau (kappa_i + kappa_j).  kind 1: |P_S|^-1 weight, 2: 2x2 solve of
// P_S, 3: P_MS^-1 weight.
__device__ __forceinline__ float2 pointwise(int kind, float2 Cr, float2 Cq, float2 mr, float c, float a2, float alpha) {
  if (kind == PK_PS) {
    const float2 lam = make_float2(mr.x + c, mr.y);
    const float2 F1 = cscale(cadd(Cr, Cq), 0.5f);
    const float2 F2 = cmul_mi(cscale(csub(Cr, Cq), 0.5f));
    const float inv = 1.0f / (lam.x * lam.x + lam.y * lam.y + a2);
    const float2 U1 = cscale(cadd(cmul(cconj(lam), F1), cscale(F2, alpha)), inv);
    const float2 U2 = cscale(csub(cmul(lam, F2), cscale(F1, alpha)), inv);
    return cadd(U1, cmul_pi(U2));
  }
  float w;
  if (kind == PK_ABS_PS) {
    const float lx = mr.x + c;
    w = rsqrtf(lx * lx + mr.y * mr.y + a2);
  } else {
    w = 1.0f / (sqrtf(mr.x * mr.x + mr.y * mr.y + a2) + c);
  }
  return cscale(Cr, w);
}

// ------------------------------------------------------------------------------------------
// Time pass: forward DFT of (half0 + i half1) * exp(-i pi t/n), pointwise solve on the frequency
// pairs (r, n-1-r), inverse DFT, unscale.  In place on the FP32 scratch; n = 32 P.  Each group
// of P lanes exchanges through its own line's tile row (the line sits in registers meanwhile),
// so a block holds the tables and NS tile stages only: two blocks per SM.
// ------------------------------------------------------------------------------------------
template <int P, int NS>
__global__ void __launch_bounds__(kThreads, 2)
    k_time_pipe(const Geom* __restrict__ G, const int* __restrict__ off, int count, Sel sel, int kind, int tot) {
  constexpr int n = 32 * P, LPB = kThreads / P;
  constexpr int PITCH = pitch_for<P>(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* tw3 = tw2 + n;
  float2* pre = tw3 + n;
  float2* mus = pre + n;                   // lambda(S_n) of the current instance
  float2* stages = mus + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const Geom& g0 = G[table_inst(off, count, sel)];
  fill_twiddles<P>(tw2, tw3, g0.twt_f);
  for (int k = tid; k < n; k += kThreads) pre[k] = __ldg(&g0.pre_f[k]);
  int mu_inst = -1;

  auto issue = [&](int tile, int st) {
    if (tile >= tot) return;
    const int inst = find_inst(off, count, tile);
    if (sel.skip(inst)) return;
    const Geom& g = G[inst];
    const int c0 = (tile - off[inst]) * LPB;
    const int l = tid % LPB;
    const bool cv = c0 + l < g.mp;
    const float* y = (const float*)g.scratch + (cv ? c0 + l : 0);
    const long long m = g.mp, mn = (long long)g.n * g.mp;
    float2* d = stages + (size_t)st * LPB * PITCH + l * PITCH;
    for (int tt = tid / LPB; tt < n; tt += kThreads / LPB) {
      cp_async<4>(&d[tt].x, y + tt * m, cv);
      cp_async<4>(&d[tt].y, y + mn + tt * m, cv);
    }
  };

#pragma unroll
  for (int s = 0; s < NS; ++s) {
    issue(blockIdx.x + s * gridDim.x, s);
    cp_commit();
  }
  const int t = lane % P;
  const int lw = warp * (32 / P) + lane / P;
  const float scale = 1.0f / (float)n;

  int it = 0;
  for (int tile = blockIdx.x; tile < tot; tile += gridDim.x, ++it) {
    const int st = it % NS;
    cp_wait<NS - 1>();
    __syncthreads();
    const int inst = find_inst(off, count, tile);
    const bool on = !sel.skip(inst);
    const Geom& g = G[inst];
    const int c0 = (tile - off[inst]) * LPB;
    float2* buf = stages + (size_t)st * LPB * PITCH;
    if (on && inst != mu_inst) {       // block-uniform
      for (int k = tid; k < n; k += kThreads) mus[k] = __ldg(&g.mu_f[k]);
      mu_inst = inst;
      __syncthreads();
    }
    if (on) {
      float2* ln = buf + lw * PITCH;
      float2 x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) x[q] = cmul(ln[t + P * q], pre[t + P * q]);
      __syncwarp();                          // the group's row is free: it serves as exchange space
      fwd2<P>(x, t, ln, tw2);
      // pointwise solve at r = t + P j; the partner n-1-r is lane P-1-t, register 31-j
      const long long col = min((long long)(c0 + lw), g.mp - 1);   // padded columns compute junk
      const int jj = (int)(col / g.lr), ii = min((int)(col - (long long)jj * g.lr), g.N - 1);
      const float c = (float)(g.tau * (__ldg(&g.kap[ii]) + __ldg(&g.kap[jj])));
      const float a2 = (float)(g.alpha * g.alpha), alpha = (float)g.alpha;
      if (kind == PK_PS) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jb = 31 - j;
          const float2 va = x[Two<P>::outreg(j)], vb = x[Two<P>::outreg(jb)];
          float2 ra, rb;                       // partner's X at n-1-r for r = t+Pj and t+P jb
          ra.x = __shfl_xor_sync(0xffffffffu, vb.x, P - 1);
          ra.y = __shfl_xor_sync(0xffffffffu, vb.y, P - 1);
          rb.x = __shfl_xor_sync(0xffffffffu, va.x, P - 1);
          rb.y = __shfl_xor_sync(0xffffffffu, va.y, P - 1);
          x[Two<P>::outreg(j)] = pointwise(PK_PS, va, cconj(ra), mus[t + P * j], c, a2, alpha);
          x[Two<P>::outreg(jb)] = pointwise(PK_PS, vb, cconj(rb), mus[t + P * jb], c, a2, alpha);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          x[Two<P>::outreg(j)] = pointwise(kind, x[Two<P>::outreg(j)], x[Two<P>::outreg(j)], mus[t + P * j], c, a2,
                                           alpha);
      }
      inv2<P>(x, t, ln, tw3);
#pragma unroll
      for (int q = 0; q < 32; ++q) ln[t + P * q] = cscale(cmulc(x[pos<32>(q)], pre[t + P * q]), scale);
    }
    __syncthreads();
    if (on) {
      const int l = tid % LPB;
      if (c0 + l < g.mp) {
        float* y = (float*)g.scratch + c0 + l;
        const long long m = g.mp, mn = (long long)g.n * g.mp;
        const float2* srcl = buf + l * PITCH;
        for (int tt = tid / LPB; tt < n; tt += kThreads / LPB) {
          const float2 v = srcl[tt];
          y[tt * m] = v.x;
          y[mn + tt * m] = v.y;
        }
      }
    }
    __syncthreads();
    issue(tile + NS * gridDim.x, st);
    cp_commit();
  }
  cp_wait<0>();
}


// ------------------------------------------------------------------------------------------
// Time pass for a general zeta (omega = exp(i zeta) other than -1) with the pipelined line FFT.
// The two halves of a spatial column are separate complex lines v_h(t) exp(-i zeta t/n); they
// sit in the adjacent lane groups 2l and 2l + 1 of a warp (P <= 16), which meet through one
// shuffle per slot for the 2x2 solve of P_S (slot r of both lines has the same frequency
// psi_r = -(zeta + 2 pi r)/n).  The result is the real part of each inverse line (Re(P^-1) on
// real vectors).  MODE 0: tiles of LPB / 2 columns of buffer 0, in place; two blocks per SM.
// ------------------------------------------------------------------------------------------
// MODE 1 (n = 512, after the time-major hand-off of pass 2): tiles of CPB spatial points
// (r, p0 .. p0+CPB-1); each line (point, half) is contiguous in buffer 1 and comes in with 16-byte
// copies; the result goes to buffer 0 in the row layout of pass 4 (value (t, r, p) at
// t mp + r lr + p), as the zeta = pi kernel does.
template <int P, int MODE = 0>
__global__ void __launch_bounds__(kThreads, 2)
    k_time_gz(const Geom* __restrict__ G, const int* __restrict__ off, int count, Sel sel, int kind, int tot) {
  static_assert(P <= 16, "the two halves of a column share one warp");
  static_assert(MODE == 0 || P == 16, "the time-major hand-off serves n = 512");
  constexpr int n = 32 * P, LPB = kThreads / P, CPB = LPB / 2;
  constexpr int PITCH = pitch_for<P>(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* tw3 = tw2 + n;
  float2* pre = tw3 + n;
  float2* mus = pre + n;                   // lambda(S_n) of the current instance
  float2* rows = mus + n;                  // row 2 l + h: column c0 + l, half h (n floats, then exchange)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const Geom& g0 = G[table_inst(off, count, sel)];
  fill_twiddles<P>(tw2, tw3, g0.twt_f);
  for (int k = tid; k < n; k += kThreads) pre[k] = __ldg(&g0.pre_f[k]);
  int mu_inst = -1;

  // MODE 1: the tile's row r and first point p0
  auto rowpt = [&](const Geom& g, int lt, int& r, int& p0) {
    const int nbs = (g.N + CPB - 1) / CPB;
    r = lt / nbs;
    p0 = (lt - r * nbs) * CPB;
  };
  // MODE 0: element e of a tile: column c0 + e % CPB, half / time (e / CPB) = h n + tt
  auto issue = [&](int tile) {
    if (tile >= tot) return;
    const int inst = find_inst(off, count, tile);
    if (sel.skip(inst)) return;
    const Geom& g = G[inst];
    if (MODE == 1) {
      int r, p0;
      rowpt(g, tile - off[inst], r, p0);
      const long long hs = (long long)g.n * g.m;
      constexpr int CH = n / 4;                // 16-byte pieces of a line
      for (int e = tid; e < 2 * CPB * CH; e += kThreads) {
        const int line = e / CH, c = e - line * CH, cl = line >> 1, h = line & 1;
        if (p0 + cl >= g.N) continue;          // points past the row compute junk that is not stored
        const float* y = (const float*)g.scratch + 2LL * g.n * g.mp + h * hs + ((long long)r * g.N + p0 + cl) * n;
        const unsigned sa = (unsigned)__cvta_generic_to_shared((float*)(rows + line * PITCH) + 4 * c);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(y + 4 * c) : "memory");
      }
      return;
    }
    const int c0 = (tile - off[inst]) * CPB;
    const long long m = g.mp, mn = (long long)g.n * g.mp;
    for (int e = tid; e < 2 * n * CPB; e += kThreads) {
      const int cl = e % CPB, rest = e / CPB, h = rest / n, tt = rest - h * n;
      const bool cv = c0 + cl < g.mp;
      const float* y = (const float*)g.scratch + h * mn + tt * m + (cv ? c0 + cl : 0);
      cp_async<4>((float*)(rows + (2 * cl + h) * PITCH) + tt, y, cv);
    }
  };

  issue(blockIdx.x);
  cp_commit();
  const int t = lane % P;
  const int lw = warp * (32 / P) + lane / P, cl = lw >> 1, h = lw & 1;
  const float scale = 1.0f / (float)n;

  for (int tile = blockIdx.x; tile < tot; tile += gridDim.x) {
    cp_wait<0>();
    __syncthreads();
    const int inst = find_inst(off, count, tile);
    const bool on = !sel.skip(inst);
    const Geom& g = G[inst];
    const int c0 = (tile - off[inst]) * CPB;
    if (on && inst != mu_inst) {       // block-uniform
      for (int k = tid; k < n; k += kThreads) mus[k] = __ldg(&g.mu_f[k]);
      mu_inst = inst;
      __syncthreads();
    }
    if (on) {
      float2* ln = rows + lw * PITCH;
      float* raw = (float*)ln;
      float2 x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) x[q] = cscale(pre[t + P * q], raw[t + P * q]);
      __syncwarp();                          // the row is free: it serves as exchange space
      fwd2<P>(x, t, ln, tw2);
      int jj, ii;
      if (MODE == 1) {
        int r, p0;
        rowpt(g, tile - off[inst], r, p0);
        jj = r;
        ii = min(p0 + cl, g.N - 1);                                   // points past N compute junk
      } else {
        const long long col = min((long long)(c0 + cl), g.mp - 1);    // padded columns compute junk
        jj = (int)(col / g.lr);
        ii = min((int)(col - (long long)jj * g.lr), g.N - 1);
      }
      const float c = (float)(g.tau * (__ldg(&g.kap[ii]) + __ldg(&g.kap[jj])));
      const float a2 = (float)(g.alpha * g.alpha), alpha = (float)g.alpha;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float2 v = x[Two<P>::outreg(j)];
        const float2 mr = mus[t + P * j];
        if (kind == PK_PS) {
          float2 o;                            // the other half's value at the same slot
          o.x = __shfl_xor_sync(0xffffffffu, v.x, P);
          o.y = __shfl_xor_sync(0xffffffffu, v.y, P);
          const float2 V1 = h ? o : v, V2 = h ? v : o;
          const float2 lam = make_float2(mr.x + c, mr.y);
          const float inv = 1.0f / (lam.x * lam.x + lam.y * lam.y + a2);
          const float2 U = h ? csub(cmul(lam, V2), cscale(V1, alpha)) : cadd(cmul(cconj(lam), V1), cscale(V2, alpha));
          x[Two<P>::outreg(j)] = cscale(U, inv);
        } else {
          float w;
          if (kind == PK_ABS_PS) {
            const float lx = mr.x + c;
            w = rsqrtf(lx * lx + mr.y * mr.y + a2);
          } else {
            w = 1.0f / (sqrtf(mr.x * mr.x + mr.y * mr.y + a2) + c);
          }
          x[Two<P>::outreg(j)] = cscale(v, w);
        }
      }
      inv2<P>(x, t, ln, tw3);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const float2 z = x[pos<32>(q)], pq = pre[t + P * q];
        raw[t + P * q] = (z.x * pq.x + z.y * pq.y) * scale;      // Re(z conj(pre)) / n
      }
    }
    __syncthreads();
    if (on) {
      const long long m = g.mp, mn = (long long)g.n * g.mp;
      int base = c0, lim = (int)min((long long)CPB, g.mp - c0);      // MODE 0: columns c0 ..
      if (MODE == 1) {
        int r, p0;
        rowpt(g, tile - off[inst], r, p0);
        base = r * g.lr + p0;                                         // MODE 1: row r, points p0 ..
        lim = min(CPB, g.N - p0);
      }
      for (int e = tid; e < 2 * n * CPB; e += kThreads) {
        const int el = e % CPB, rest = e / CPB, hh = rest / n, tt = rest - hh * n;
        if (el < lim)
          ((float*)g.scratch)[hh * mn + tt * m + base + el] = ((const float*)(rows + (2 * el + hh) * PITCH))[tt];
      }
    }
    __syncthreads();
    issue(tile + gridDim.x);
    cp_commit();
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Time pass for n = 512 with one line per warp: lane t holds x[t + 32 q] (16 values).
//   forward: 16-point register DFT over q, twiddle W_512^{t k1}, exchange through the line's own
//   tile row (row k1, column t XOR k1), then lane (k1, h) = (u mod 16, u / 16) runs a 16-point
//   DFT over t'' of V[2t''+h][k1] and one radix-2 step across lanes u, u^16:
//       X[k1 + 16 k2 + 256 h] = G_0[k2] + (-1)^h W_32^{k2} G_1[k2].
//   The partner slot n-1-r of r = k1 + 16 k2 + 256 h is lane u^31, register 15-k2.
// Tiles of 8 columns come in through NS cp.async stages; two blocks run per SM.
// ------------------------------------------------------------------------------------------
// MODE 0: tiles of 8 spatial columns of buffer 0 (any layout), strided loads, result in place.
// MODE 1: tiles of 8 spatial points (r, p0 .. p0+7) of the time-major buffer 1 (contiguous time
// lines, 16-byte copies), result written to buffer 0 in the row layout of pass 4 (value
// (t, r, p) at t mp + r lr + p): row segments of 8 values.
// MINB: resident blocks per SM the compiler budgets registers for (2: 128 registers a thread, with
// NS = 2 tile stages; 3 or 4: at most 85 or 64 registers and one stage, the extra blocks hiding
// the loads).
template <int NS, int MODE, int MINB = 2>
__global__ void __launch_bounds__(kThreads, MINB)
    k_time512(const Geom* __restrict__ G, const int* __restrict__ off, int count, Sel sel, int kind, int tot) {
  constexpr int n = 512, LPB = kWarps;
  constexpr int PITCH = pitch_for<32>(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw1 = (float2*)smem_raw;        // [k1 * 32 + t] = W_512^{t k1}, k1 < 16
  float2* tw32 = tw1 + n;                  // [h * 16 + k] = W_32^{h k}
  float2* pre = tw32 + 32;                 // exp(-i pi t / n)
  float2* mus = pre + n;                   // lambda(S_n) of the current instance
  float2* stages = mus + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    const Geom& g0 = G[table_inst(off, count, sel)];
    const float2* __restrict__ w = g0.twt_f;
    for (int k = tid; k < n; k += kThreads) {
      tw1[k] = __ldg(&w[(k % 32) * (k / 32)]);
      pre[k] = __ldg(&g0.pre_f[k]);
    }
    if (tid < 32) tw32[tid] = __ldg(&w[16 * (tid / 16) * (tid % 16)]);
  }

  auto issue = [&](int tile, int st) {
    if (tile >= tot) return;
    const int inst = find_inst(off, count, tile);
    if (sel.skip(inst)) return;
    const Geom& g = G[inst];
    if (MODE == 0) {
      const int c0 = (tile - off[inst]) * LPB;
      const int l = tid % LPB;
      const bool cv = c0 + l < g.mp;
      const float* y = (const float*)g.scratch + (cv ? c0 + l : 0);
      const long long m = g.mp, mn = (long long)g.n * g.mp;
      float2* d = stages + (size_t)st * LPB * PITCH + l * PITCH;
      for (int tt = tid / LPB; tt < n; tt += kThreads / LPB) {
        cp_async<4>(&d[tt].x, y + tt * m, cv);
        cp_async<4>(&d[tt].y, y + mn + tt * m, cv);
      }
    } else {
      // each warp copies its own time line: re[512] then im[512] (raw floats) into its tile row
      const int lt = tile - off[inst], nbs = (g.N + LPB - 1) / LPB;
      const int r = lt / nbs, p = (lt - r * nbs) * LPB + warp;
      if (p < g.N) {
        const float* y = (const float*)g.scratch + 2LL * g.n * g.mp + ((long long)r * g.N + p) * n;
        const long long hs = (long long)g.n * g.m;
        float* d = (float*)(stages + (size_t)st * LPB * PITCH + warp * PITCH);
#pragma unroll
        for (int h = 0; h < 2; ++h)
          for (int c = lane; c < n / 4; c += 32) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(d + h * n + 4 * c);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(y + h * hs + 4 * c) : "memory");
          }
      }
    }
  };
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    issue(blockIdx.x + s * gridDim.x, s);
    cp_commit();
  }
  const int t = lane, k1 = lane & 15, h = lane >> 4;
  const float sg = h ? -1.f : 1.f;
  const float scale = 1.0f / (float)n;
  int mu_inst = -1;

  int it = 0;
  for (int tile = blockIdx.x; tile < tot; tile += gridDim.x, ++it) {
    const int st = it % NS;
    cp_wait<NS - 1>();
    __syncthreads();
    const int inst = find_inst(off, count, tile);
    const bool on = !sel.skip(inst);
    const Geom& g = G[inst];
    const int c0 = (tile - off[inst]) * LPB;
    if (on && inst != mu_inst) {       // block-uniform
      for (int k = tid; k < n; k += kThreads) mus[k] = __ldg(&g.mu_f[k]);
      mu_inst = inst;
      __syncthreads();
    }
    float2* buf = stages + (size_t)st * LPB * PITCH;
    if (on) {
      float2* ln = buf + warp * PITCH;
      float2 x[16];
      if (MODE == 0) {
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = cmul(ln[t + 32 * q], pre[t + 32 * q]);
      } else {
        const float* raw = (const float*)ln;
#pragma unroll
        for (int q = 0; q < 16; ++q) x[q] = cmul(make_float2(raw[t + 32 * q], raw[n + t + 32 * q]), pre[t + 32 * q]);
      }
      reg_dft<float2, float, 16>(x, false);
      __syncwarp();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        float2 v = x[pos<16>(kk)];
        if (kk) v = cmul(v, tw1[kk * 32 + t]);
        ln[kk * 32 + (t ^ kk)] = v;
      }
      __syncwarp();
#pragma unroll
      for (int t2 = 0; t2 < 16; ++t2) x[t2] = ln[k1 * 32 + ((2 * t2 + h) ^ k1)];
      reg_dft<float2, float, 16>(x, false);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        float2 v = x[pos<16>(k2)];
        if (k2) v = cmul(v, tw32[h * 16 + k2]);
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, 16);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, 16);
        x[pos<16>(k2)] = make_float2(fmaf(sg, v.x, o.x), fmaf(sg, v.y, o.y));
      }
      // pointwise solve at r = k1 + 16 k2 + 256 h
      int jj, ii;
      if (MODE == 0) {
        const long long col = min((long long)(c0 + warp), g.mp - 1);  // padded columns compute junk
        jj = (int)(col / g.lr);
        ii = min((int)(col - (long long)jj * g.lr), g.N - 1);
      } else {
        const int lt = tile - off[inst], nbs = (g.N + LPB - 1) / LPB;
        jj = lt / nbs;
        ii = min((lt - jj * nbs) * LPB + warp, g.N - 1);               // points past N compute junk
      }
      const float c = (float)(g.tau * (__ldg(&g.kap[ii]) + __ldg(&g.kap[jj])));
      const float a2 = (float)(g.alpha * g.alpha), alpha = (float)g.alpha;
      if (kind == PK_PS) {
#pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
          const int kb = 15 - k2;
          const float2 va = x[pos<16>(k2)], vb = x[pos<16>(kb)];
          float2 ra, rb;                    // the partner's coefficients at n-1-r
          ra.x = __shfl_xor_sync(0xffffffffu, vb.x, 31);
          ra.y = __shfl_xor_sync(0xffffffffu, vb.y, 31);
          rb.x = __shfl_xor_sync(0xffffffffu, va.x, 31);
          rb.y = __shfl_xor_sync(0xffffffffu, va.y, 31);
          x[pos<16>(k2)] = pointwise(PK_PS, va, cconj(ra), mus[k1 + 16 * k2 + 256 * h], c, a2, alpha);
          x[pos<16>(kb)] = pointwise(PK_PS, vb, cconj(rb), mus[k1 + 16 * kb + 256 * h], c, a2, alpha);
        }
      } else {
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2)
          x[pos<16>(k2)] = pointwise(kind, x[pos<16>(k2)], x[pos<16>(k2)], mus[k1 + 16 * k2 + 256 * h], c, a2, alpha);
      }
      // inverse: undo the radix-2 step, W_32 twiddle, 16-point DFT over k2, exchange back,
      // W_512 twiddle, 16-point DFT over k1, unscale
      float2 z[16];
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) {
        const float2 v = x[pos<16>(k2)];
        float2 o;
        o.x = __shfl_xor_sync(0xffffffffu, v.x, 16);
        o.y = __shfl_xor_sync(0xffffffffu, v.y, 16);
        float2 a = make_float2(fmaf(sg, v.x, o.x), fmaf(sg, v.y, o.y));
        if (k2) a = cmulc(a, tw32[h * 16 + k2]);
        z[k2] = a;
      }
      reg_dft<float2, float, 16>(z, true);
#pragma unroll
      for (int t2 = 0; t2 < 16; ++t2) ln[k1 * 32 + ((2 * t2 + h) ^ k1)] = z[pos<16>(t2)];
      __syncwarp();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        float2 v = ln[kk * 32 + (t ^ kk)];
        if (kk) v = cmulc(v, tw1[kk * 32 + t]);
        x[kk] = v;
      }
      reg_dft<float2, float, 16>(x, true);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 16; ++q) ln[t + 32 * q] = cscale(cmulc(x[pos<16>(q)], pre[t + 32 * q]), scale);
    }
    __syncthreads();
    if (on && MODE == 0) {
      const int l = tid % LPB;
      if (c0 + l < g.mp) {
        float* y = (float*)g.scratch + c0 + l;
        const long long m = g.mp, mn = (long long)g.n * g.mp;
        const float2* srcl = buf + l * PITCH;
        for (int tt = tid / LPB; tt < n; tt += kThreads / LPB) {
          const float2 v = srcl[tt];
          y[tt * m] = v.x;
          y[mn + tt * m] = v.y;
        }
      }
    } else if (on) {
      const int l = tid % LPB;
      const int lt = tile - off[inst], nbs = (g.N + LPB - 1) / LPB;
      const int r = lt / nbs, p = (lt - r * nbs) * LPB + l;
      if (p < g.N) {
        float* y = (float*)g.scratch + (long long)r * g.lr + p;
        const long long m = g.mp, mn = (long long)g.n * g.mp;
        const float2* srcl = buf + l * PITCH;
        for (int tt = tid / LPB; tt < n; tt += kThreads / LPB) {
          const float2 v = srcl[tt];
          y[tt * m] = v.x;
          y[mn + tt * m] = v.y;
        }
      }
    }
    __syncthreads();
    issue(tile + NS * gridDim.x, st);
    cp_commit();
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
constexpr int kNsTime = 2;
constexpr int kNsTimePipe = 1;     // k_time_pipe: the second resident block hides the tile loads

template <int P>
size_t dst_tables_smem() { return (size_t)(32 * P + P + kWarps * odd_scratch_per_warp<P>()) * sizeof(float2); }
template <typename TIn, int P, bool EV>
size_t dst_rows_smem() {
  return dst_tables_smem<P>() + (size_t)kThreads / P * 2 * row_slot_elems<TIn>(line_values<P, EV>()) * sizeof(TIn);
}
template <typename TIn, int P, bool EV>
size_t dst_rowsT_smem() {
  return (size_t)(32 * P + P + kWarps * rowsT_region<P>()) * sizeof(float2) +
         (size_t)kThreads / P * 2 * row_slot_elems<TIn>(line_values<P, EV>()) * sizeof(TIn);
}
template <int P>
size_t time_smem() {     // twiddles, D_omega weights, lambda(S_n), tile stages
  return (size_t)(4 * 32 * P) * sizeof(float2) +
         (size_t)kNsTimePipe * (kThreads / P) * pitch_for<P>(32 * P) * sizeof(float2);
}
size_t time512_smem(int ns = kNsTime) { return (size_t)(3 * 512 + 32 + ns * kWarps * pitch_for<32>(512)) * sizeof(float2); }

// Launch a persistent kernel: at most as many blocks as fit on the device at once.  The figure
// (and the shared-memory limit it needs) is set up once per kernel and device; `resident` keeps it.
template <typename K, typename... Args>
cudaError_t launch_persistent(K kern, size_t smem, int tot, DeviceInt& resident, cudaStream_t st, Args... args) {
  if (tot <= 0) return cudaSuccess;
  int res = 0;
  cudaError_t e = resident.get(&res, [&](int* out) {
    cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e2 != cudaSuccess) return e2;
    int occ = 0, dev = 0, sms = 0;
    if ((e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem)) != cudaSuccess) return e2;
    if ((e2 = cudaGetDevice(&dev)) != cudaSuccess) return e2;
    if ((e2 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e2;
    *out = std::max(1, occ) * std::max(1, sms);
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  kern<<<std::min(tot, res), kThreads, smem, st>>>(args...);
  return cudaGetLastError();
}

template <typename TIn, typename TOut, int P, bool EV>
cudaError_t launch_rows(const Batch& B, int in_sel, int out_sel, int inv) {
  static DeviceInt resident;
  return launch_persistent(k_dst_rows<TIn, TOut, P, EV>, dst_rows_smem<TIn, P, EV>(), B.tot_dst_i[1], resident,
                           B.stream, B.G, (const Slots*)B.S, B.off_dst_i[1], B.count, B.sel(), in_sel, out_sel,
                           B.tot_dst_i[1], inv);
}

template <typename TIn, int P, int MODE, bool EV>
cudaError_t launch_rowsT(const Batch& B, int in_sel, int out_sel, int inv) {
  static DeviceInt resident;
  // MODE 0 tiles: (time step, LPB rows) -> dst_j offsets; MODE 1 tiles: (row, LPB time steps),
  // as many as the contiguous-line tiles -> dst_i offsets
  const int* off = MODE == 0 ? B.off_dst_j[1] : B.off_dst_i[1];
  const int tot = MODE == 0 ? B.tot_dst_j[1] : B.tot_dst_i[1];
  return launch_persistent(k_dst_rowsT<TIn, P, MODE, EV>, dst_rowsT_smem<TIn, P, EV>(), tot, resident, B.stream,
                           B.G, (const Slots*)B.S, off, B.count, B.sel(), in_sel, out_sel, tot, inv);
}

template <int P>
cudaError_t launch_time(const Batch& B, int kind, bool time_major = false) {
  static DeviceInt resident;
  if (P == 16) {
    static DeviceInt resident512[6];
    if (B.t512v == 1) {     // the autotuner's variants: one tile stage, three or four blocks per SM
      if (time_major)
        return launch_persistent(k_time512<1, 1, 3>, time512_smem(1), B.tot_time[1], resident512[3], B.stream, B.G,
                                 B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
      return launch_persistent(k_time512<1, 0, 3>, time512_smem(1), B.tot_time[1], resident512[2], B.stream, B.G,
                               B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
    }
    if (B.t512v == 2) {
      if (time_major)
        return launch_persistent(k_time512<1, 1, 4>, time512_smem(1), B.tot_time[1], resident512[5], B.stream, B.G,
                                 B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
      return launch_persistent(k_time512<1, 0, 4>, time512_smem(1), B.tot_time[1], resident512[4], B.stream, B.G,
                               B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
    }
    if (time_major)
      return launch_persistent(k_time512<kNsTime, 1>, time512_smem(), B.tot_time[1], resident512[1], B.stream, B.G,
                               B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
    return launch_persistent(k_time512<kNsTime, 0>, time512_smem(), B.tot_time[1], resident512[0], B.stream, B.G,
                             B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
  }
  return launch_persistent(k_time_pipe<P, kNsTimePipe>, time_smem<P>(), B.tot_time[1], resident, B.stream, B.G,
                           B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
}

template <int P>
cudaError_t launch_time_gz(const Batch& B, int kind, bool time_major = false) {
  static DeviceInt resident[2];
  if constexpr (P == 16) {
    if (time_major)
      return launch_persistent(k_time_gz<16, 1>, time_smem<16>(), B.tot_time[1], resident[1], B.stream, B.G,
                               B.off_time[1], B.count, B.sel(), kind, B.tot_time[1]);
  }
  return launch_persistent(k_time_gz<P>, time_smem<P>(), B.tot_time[1], resident[0], B.stream, B.G, B.off_time[1],
                           B.count, B.sel(), kind, B.tot_time[1]);
}

// pass `stage` (1, 2, 4, 5) of the FP32 apply; scratch buffers: -1 = buffer 0, -2 = buffer 1.
// time_major: pass 2 writes time-major lines to buffer 1 and the time pass writes buffer 0 back
// in the row layout, so pass 4 finds its input where it would otherwise be.  EV: the Neumann
// route's DCT-I pair, forward in passes 1-2 and inverse in passes 4-5.
template <int P, bool EV>
cudaError_t dst_pass_p(const Batch& B, int stage, int in_slot, int out_slot, bool time_major) {
  const int inv = stage >= 4;
  switch (stage) {
    case 1: return launch_rowsT<double, P, 0, EV>(B, in_slot, -1, inv);
    case 2:
      return time_major ? launch_rowsT<float, P, 1, EV>(B, -1, -2, inv) : launch_rows<float, float, P, EV>(B, -1, -1, inv);
    case 4: return launch_rowsT<float, P, 0, EV>(B, -1, -2, inv);
    default: return launch_rows<float, double, P, EV>(B, -2, out_slot, inv);
  }
}

}  // namespace

// P of the pipelined passes for an instance (0: not eligible): DST lines of 2L = 32 P points,
// time lines of n = 32 P points, P a power of two in [2, 32] (Neumann's DCT-I lines: P >= 8);
// the constant-coefficient route only.
int pipe_time_p(const Geom& g);
int pipe_dst_p(const Geom& g) {
  // the padded scratch layout needs the pipelined time pass
  if (g.mg_route || (g.tune & TUNE_NO_PIPE_DST) || !pipe_time_p(g)) return 0;
  const int M = 2 * g.L;
  if (M % 32) return 0;
  const int P = M / 32;
  if (g.bc == PCB_BC_NEUMANN && P < 8) return 0;
  return (P >= 2 && P <= 32 && (P & (P - 1)) == 0) ? P : 0;
}
int pipe_time_p(const Geom& g) {
  if (g.mg_route || (g.tune & TUNE_NO_PIPE_TIME) || g.n % 32) return 0;
  const int P = g.n / 32;
  if (!g.zeta_pi && P > 16) return 0;        // general zeta: the two halves of a column share a warp
  return (P >= 2 && P <= 32 && (P & (P - 1)) == 0) ? P : 0;
}
// family codes: P, plus 64 when pass 2 writes time-major lines for the n = 512 time pass, plus
// 128 for the DCT-I lines of the Neumann route, plus 256 for the general-zeta time pass.  The
// time-major hand-off needs pipelined spatial and time passes at n = 512 (P = 16 in time).
static bool time_major_handoff(const Geom& g) {
  return g.n == 512 && !(g.tune & TUNE_NO_HANDOFF) && pipe_dst_p(g) && pipe_time_p(g) == 16;
}
int pipe_dst_code(const Geom& g) {
  const int p = pipe_dst_p(g);
  return p ? (p | (time_major_handoff(g) ? 64 : 0) | (g.bc == PCB_BC_NEUMANN ? 128 : 0)) : 0;
}
int pipe_time_code(const Geom& g) {
  const int p = pipe_time_p(g);
  if (!p) return 0;
  return p | (g.zeta_pi ? 0 : 256) | (time_major_handoff(g) ? 64 : 0);
}
// spatial columns per tile of the pipelined time pass (n = 512: one line per warp; general zeta:
// two lines, the halves, per column)
int pipe_time_cols(int n, int zeta_pi) {
  if (!zeta_pi) return kThreads / (n / 32) / 2;
  return n == 512 ? kWarps : kThreads / (n / 32);
}
// lines per tile of the pipelined DST passes
int pipe_dst_lines(int L) { return kThreads / (2 * L / 32); }

cudaError_t pipe_upload_constants() { return upload_w96(); }

// DST pass `stage` of the FP32 apply; B.pipe_pd is the P shared by the instances it covers.
cudaError_t pipe_dst_pass(const Batch& B, int stage, int in_slot, int out_slot) {
  const bool tm = B.pipe_pd & 64;
  if (B.pipe_pd & 128) {
    switch (B.pipe_pd & 63) {
      case 8: return dst_pass_p<8, true>(B, stage, in_slot, out_slot, tm);
      case 16: return dst_pass_p<16, true>(B, stage, in_slot, out_slot, tm);
      case 32: return dst_pass_p<32, true>(B, stage, in_slot, out_slot, tm);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (B.pipe_pd & 63) {
    case 2: return dst_pass_p<2, false>(B, stage, in_slot, out_slot, tm);
    case 4: return dst_pass_p<4, false>(B, stage, in_slot, out_slot, tm);
    case 8: return dst_pass_p<8, false>(B, stage, in_slot, out_slot, tm);
    case 16: return dst_pass_p<16, false>(B, stage, in_slot, out_slot, tm);
    case 32: return dst_pass_p<32, false>(B, stage, in_slot, out_slot, tm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t pipe_time_pass(const Batch& B, int kind) {
  const bool tm = B.pipe_pt & 64;
  if (B.pipe_pt & 256) {
    switch (B.pipe_pt & 63) {
      case 2: return launch_time_gz<2>(B, kind);
      case 4: return launch_time_gz<4>(B, kind);
      case 8: return launch_time_gz<8>(B, kind);
      case 16: return launch_time_gz<16>(B, kind, tm);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (B.pipe_pt & 63) {
    case 2: return launch_time<2>(B, kind);
    case 4: return launch_time<4>(B, kind);
    case 8: return launch_time<8>(B, kind);
    case 16: return launch_time<16>(B, kind, tm);
    case 32: return launch_time<32>(B, kind);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pcb
