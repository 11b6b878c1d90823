// Pipelined FP32 preconditioner passes for power-of-two line lengths (paper Sec. 3.5).
//
// The same five passes as precond.cu (DST-I along x1, DST-I along x2, time DFT + pointwise solve
// + inverse time DFT, DST-I along x2, DST-I along x1), organised to hide memory latency:
//   * Persistent blocks (one per SM, eight warps) walk the tiles of a pass.  The input of each
//     tile is fetched with asynchronous copies (cp.async) into one of NS shared-memory stages, so
//     the loads of the next tiles are in flight while the current tile is transformed.
//   * A line of length M = 32 P (2 <= P <= 32) is transformed by P lanes holding 32 values each,
//     as a two-stage FFT: with s = t + P q and k = k1 + 32 k2,
//         X[k1 + 32 k2] = sum_t W_P^{t k2} W_M^{t k1} sum_q x[t + P q] W_32^{q k1},
//     i.e. a 32-point register DFT per lane, the twiddle W_M^{t k1}, an exchange through a per-warp
//     shared-memory block (XOR-swizzled, free of bank conflicts) and 32/P register DFTs of size P.
//     Lane t starts with x[t + P q] and ends with X[u + P j] (u = t): both cyclic with stride P, so
//     contiguous lines load and store with coalesced accesses and no bit reversal.  The inverse
//     runs the same steps in reverse order.
// Scratch layout and the value of every pass are those of precond.cu, so the two implementations
// can be mixed pass by pass.
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

template <typename TIn> struct CxOf;
template <> struct CxOf<float> { using T = float2; };
template <> struct CxOf<double> { using T = double2; };

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// ------------------------------------------------------------------------------------------
// DST-I pass.  AXIS 0: lines along x1 (contiguous); AXIS 1: lines along x2 (stride N).
// in_slot / out_slot >= 0: FP64 vector slot; -1: the FP32 scratch.
// A tile is LPB = 256 / P lines; line length L - 1 = 16 P - 1 = N.
// ------------------------------------------------------------------------------------------
template <typename TIn, typename TOut, int P, int AXIS, int NS>
__global__ void __launch_bounds__(kThreads, 1)
    k_dst_pipe(const Geom* __restrict__ G, const Slots* __restrict__ S, const int* __restrict__ off, int count,
               Sel sel, int in_slot, int out_slot, int tot) {
  constexpr int M = 32 * P, L = 16 * P, N = L - 1, LPB = kThreads / P;
  constexpr int PITCH = pitch_for<P>(N);
  constexpr int m = N * N;
  constexpr int NBT = (N + LPB - 1) / LPB;       // x2-line tiles per time step
  using CI = typename CxOf<TIn>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* scr_all = tw2 + M;
  CI* stages = (CI*)(scr_all + kWarps * kScrWarp);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  fill_twiddles<P>(tw2, nullptr, G[table_inst(off, count, sel)].twd_f);

  // issue the asynchronous loads of tile `tile` into stage `st`
  auto issue = [&](int tile, int st) {
    if (tile >= tot) return;
    const int inst = find_inst(off, count, tile);
    if (sel.skip(inst)) return;
    const Geom& g = G[inst];
    const int lt = tile - off[inst];
    const long long mn = g.mn;
    const TIn* in = in_slot >= 0 ? (const TIn*)S[inst].v[in_slot] : (const TIn*)g.scratch;
    CI* buf = stages + (size_t)st * LPB * PITCH;
    if (AXIS == 0) {
      const long long nlines = (long long)g.n * N;
      for (int l = warp; l < LPB; l += kWarps) {
        const long long line = (long long)lt * LPB + l;
        const bool lv = line < nlines;
        const TIn* src = in + (lv ? line : 0) * N;
        CI* d = buf + l * PITCH;
        for (int q = lane; q < N; q += 32) {
          cp_async<sizeof(TIn)>(&d[q].x, src + q, lv);
          cp_async<sizeof(TIn)>(&d[q].y, src + mn + q, lv);
        }
      }
    } else {
      const int t0 = lt / NBT, i0 = (lt - t0 * NBT) * LPB;
      const int l = tid % LPB;
      const bool iv = i0 + l < N;
      const TIn* src = in + (long long)t0 * m + (iv ? i0 + l : 0);
      CI* d = buf + l * PITCH;
      for (int q = tid / LPB; q < N; q += kThreads / LPB) {
        cp_async<sizeof(TIn)>(&d[q].x, src + (long long)q * N, iv);
        cp_async<sizeof(TIn)>(&d[q].y, src + mn + (long long)q * N, iv);
      }
    }
  };

#pragma unroll
  for (int s = 0; s < NS; ++s) {
    issue(blockIdx.x + s * gridDim.x, s);
    cp_commit();
  }
  const float sc = __frsqrt_rn((float)(2 * L));     // DST-I normalisation 0.5 sqrt(2/L)
  float2* scr = scr_all + warp * kScrWarp + (lane / P) * (32 * P + P);
  const int t = lane % P;
  const int lw = warp * (32 / P) + lane / P;      // this lane group's line within the tile

  int it = 0;
  for (int tile = blockIdx.x; tile < tot; tile += gridDim.x, ++it) {
    const int st = it % NS;
    cp_wait<NS - 1>();
    __syncthreads();
    const int inst = find_inst(off, count, tile);
    const bool on = !sel.skip(inst);
    const Geom& g = G[inst];
    const int lt = tile - off[inst];
    const long long mn = g.mn;
    CI* buf = stages + (size_t)st * LPB * PITCH;
    bool lv;
    long long line = 0;
    int t0 = 0, i0 = 0;
    if (AXIS == 0) {
      line = (long long)lt * LPB + lw;
      lv = on && line < (long long)g.n * N;
    } else {
      t0 = lt / NBT;
      i0 = (lt - t0 * NBT) * LPB;
      lv = on && i0 + lw < N;
    }
    if (on) {
      // gather the odd extension: z_s = x_{s-1} (1 <= s <= N), -x_{M-s-1} (L < s < M), 0 else
      const CI* ln = buf + lw * PITCH;
      float2 x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int s = t + P * q;
        float2 v;
        if (q < 16) {
          v = to_f2(ln[s > 0 ? s - 1 : 0]);
          if (s == 0) v = make_float2(0.f, 0.f);
        } else {
          v = to_f2(ln[s > L ? M - s - 1 : 0]);
          v.x = -v.x; v.y = -v.y;
          if (s == L) v = make_float2(0.f, 0.f);
        }
        x[q] = v;
      }
      fwd2<P>(x, t, scr, tw2);
      // outputs p = t + P j, 1 <= p <= N (j < 16): S_p = (i/2) sqrt(2/L) Y_p
      if (AXIS == 0) {
        if (lv) {
          TOut* out = out_slot >= 0 ? (TOut*)S[inst].v[out_slot] : (TOut*)g.scratch;
          TOut* d = out + line * N;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int p = t + P * j;
            const float2 Y = x[Two<P>::outreg(j)];
            if (p >= 1) {
              d[p - 1] = (TOut)(-Y.y * sc);
              d[mn + p - 1] = (TOut)(Y.x * sc);
            }
          }
        }
      } else {
        CI* lnw = buf + lw * PITCH;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int p = t + P * j;
          const float2 Y = x[Two<P>::outreg(j)];
          if (p >= 1) {
            CI v;
            v.x = -Y.y * sc;
            v.y = Y.x * sc;
            lnw[p - 1] = v;
          }
        }
      }
    }
    __syncthreads();
    if (AXIS == 1 && on) {
      TOut* out = out_slot >= 0 ? (TOut*)S[inst].v[out_slot] : (TOut*)g.scratch;
      const int l = tid % LPB;
      if (i0 + l < N) {
        TOut* d = out + (long long)t0 * m + i0 + l;
        const CI* srcl = buf + l * PITCH;
        for (int q = tid / LPB; q < N; q += kThreads / LPB) {
          const CI v = srcl[q];
          d[(long long)q * N] = (TOut)v.x;
          d[mn + (long long)q * N] = (TOut)v.y;
        }
      }
      __syncthreads();
    }
    issue(tile + NS * gridDim.x, st);
    cp_commit();
  }
  cp_wait<0>();
}

// ------------------------------------------------------------------------------------------
// Time pass: forward DFT of (half0 + i half1) * exp(-i pi t/n), pointwise solve on the frequency
// pairs (r, n-1-r), inverse DFT, unscale.  In place on the FP32 scratch; n = 32 P.
// ------------------------------------------------------------------------------------------
template <int P, int NS>
__global__ void __launch_bounds__(kThreads, 1)
    k_time_pipe(const Geom* __restrict__ G, const int* __restrict__ off, int count, Sel sel, int kind, int tot) {
  constexpr int n = 32 * P, LPB = kThreads / P;
  constexpr int PITCH = pitch_for<P>(n);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw2 = (float2*)smem_raw;
  float2* tw3 = tw2 + n;
  float2* pre = tw3 + n;
  float2* scr_all = pre + n;
  float2* stages = scr_all + kWarps * kScrWarp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  const Geom& g0 = G[table_inst(off, count, sel)];
  fill_twiddles<P>(tw2, tw3, g0.twt_f);
  for (int k = tid; k < n; k += kThreads) pre[k] = __ldg(&g0.pre_f[k]);

  auto issue = [&](int tile, int st) {
    if (tile >= tot) return;
    const int inst = find_inst(off, count, tile);
    if (sel.skip(inst)) return;
    const Geom& g = G[inst];
    const int c0 = (tile - off[inst]) * LPB;
    const int l = tid % LPB;
    const bool cv = c0 + l < g.m;
    const float* y = (const float*)g.scratch + (cv ? c0 + l : 0);
    const long long m = g.m, mn = g.mn;
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
  float2* scr = scr_all + warp * kScrWarp + (lane / P) * (32 * P + P);
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
    if (on) {
      float2* ln = buf + lw * PITCH;
      float2 x[32];
#pragma unroll
      for (int q = 0; q < 32; ++q) x[q] = cmul(ln[t + P * q], pre[t + P * q]);
      fwd2<P>(x, t, scr, tw2);
      // pointwise solve at r = t + P j; the partner n-1-r is lane P-1-t, register 31-j
      const int col = min(c0 + lw, g.m - 1);
      const int jj = col / g.N, ii = col - jj * g.N;
      const float c = (float)(g.tau * (__ldg(&g.kap[ii]) + __ldg(&g.kap[jj])));
      const float a2 = (float)(g.alpha * g.alpha), alpha = (float)g.alpha;
      const float2* __restrict__ mu = g.mu_f;
      if (kind == PK_PS) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int jb = 31 - j;
          float2 va = x[Two<P>::outreg(j)], vb = x[Two<P>::outreg(jb)];
          float2 ra, rb;                       // partner's X at n-1-r for r = t+Pj and t+P jb
          ra.x = __shfl_xor_sync(0xffffffffu, vb.x, P - 1);
          ra.y = __shfl_xor_sync(0xffffffffu, vb.y, P - 1);
          rb.x = __shfl_xor_sync(0xffffffffu, va.x, P - 1);
          rb.y = __shfl_xor_sync(0xffffffffu, va.y, P - 1);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int jx = h ? jb : j;
            const float2 Cr = h ? vb : va;
            const float2 Cq = cconj(h ? rb : ra);
            const float2 mr = __ldg(&mu[t + P * jx]);
            const float2 lam = make_float2(mr.x + c, mr.y);
            const float2 F1 = cscale(cadd(Cr, Cq), 0.5f);
            const float2 F2 = cmul_mi(cscale(csub(Cr, Cq), 0.5f));
            const float inv = 1.0f / (lam.x * lam.x + lam.y * lam.y + a2);
            const float2 U1 = cscale(cadd(cmul(cconj(lam), F1), cscale(F2, alpha)), inv);
            const float2 U2 = cscale(csub(cmul(lam, F2), cscale(F1, alpha)), inv);
            x[Two<P>::outreg(jx)] = cadd(U1, cmul_pi(U2));
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float2 mr = __ldg(&mu[t + P * j]);
          float w;
          if (kind == PK_ABS_PS) {
            const float lx = mr.x + c;
            w = rsqrtf(lx * lx + mr.y * mr.y + a2);
          } else {
            w = 1.0f / (sqrtf(mr.x * mr.x + mr.y * mr.y + a2) + c);
          }
          x[Two<P>::outreg(j)] = cscale(x[Two<P>::outreg(j)], w);
        }
      }
      inv2<P>(x, t, scr, tw3);
#pragma unroll
      for (int q = 0; q < 32; ++q) ln[t + P * q] = cscale(cmulc(x[pos<32>(q)], pre[t + P * q]), scale);
    }
    __syncthreads();
    if (on) {
      const int l = tid % LPB;
      if (c0 + l < g.m) {
        float* y = (float*)g.scratch + c0 + l;
        const long long m = g.m, mn = g.mn;
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
constexpr int kNsDst = 3, kNsDstD = 2, kNsTime = 2;

template <int P>
size_t dst_smem(int in_bytes, int ns) {
  return (size_t)(32 * P + kWarps * kScrWarp) * sizeof(float2) +
         (size_t)ns * (kThreads / P) * pitch_for<P>(16 * P - 1) * 2 * in_bytes;
}
template <int P>
size_t time_smem(int ns) {
  return (size_t)(3 * 32 * P + kWarps * kScrWarp) * sizeof(float2) +
         (size_t)ns * (kThreads / P) * pitch_for<P>(32 * P) * sizeof(float2);
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// blocks per SM of a persistent kernel (queried once per kernel)
template <typename K>
int resident_blocks(K kernel, size_t smem, int& cache) {
  if (!cache) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, smem);
    cache = std::max(1, occ) * sm_count();
  }
  return cache;
}

template <typename TIn, typename TOut, int P, int AXIS>
cudaError_t launch_dst(const Batch& B, int in_slot, int out_slot) {
  constexpr int NS = sizeof(TIn) == 8 ? kNsDstD : kNsDst;
  auto kern = k_dst_pipe<TIn, TOut, P, AXIS, NS>;
  const size_t smem = dst_smem<P>(sizeof(TIn), NS);
  static int resident = 0;
  const int* off = AXIS == 0 ? B.off_dst_i[1] : B.off_dst_j[1];
  const int tot = AXIS == 0 ? B.tot_dst_i[1] : B.tot_dst_j[1];
  if (tot <= 0) return cudaSuccess;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = std::min(tot, resident_blocks(kern, smem, resident));
  kern<<<grid, kThreads, smem, B.stream>>>(B.G, B.S, off, B.count, B.sel(), in_slot, out_slot, tot);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_time(const Batch& B, int kind) {
  auto kern = k_time_pipe<P, kNsTime>;
  const size_t smem = time_smem<P>(kNsTime);
  static int resident = 0;
  const int tot = B.tot_time[1];
  if (tot <= 0) return cudaSuccess;
  if (!resident) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = std::min(tot, resident_blocks(kern, smem, resident));
  kern<<<grid, kThreads, smem, B.stream>>>(B.G, B.off_time[1], B.count, B.sel(), kind, tot);
  return cudaGetLastError();
}

template <int P>
cudaError_t dst_pass_p(const Batch& B, int axis, int in_slot, int out_slot) {
  if (axis == 0 && in_slot >= 0) return launch_dst<double, float, P, 0>(B, in_slot, -1);
  if (axis == 0 && out_slot >= 0) return launch_dst<float, double, P, 0>(B, -1, out_slot);
  if (axis == 0) return launch_dst<float, float, P, 0>(B, -1, -1);
  return launch_dst<float, float, P, 1>(B, -1, -1);
}

}  // namespace

// P of the pipelined passes for an instance (0: not eligible): DST lines of 2L = 32 P points,
// time lines of n = 32 P points, P a power of two in [2, 32]; the constant-coefficient route only.
int pipe_dst_p(const Geom& g) {
  if (g.var_a) return 0;
  const int M = 2 * g.L;
  if (M % 32) return 0;
  const int P = M / 32;
  return (P >= 2 && P <= 32 && (P & (P - 1)) == 0) ? P : 0;
}
int pipe_time_p(const Geom& g) {
  if (g.var_a || g.n % 32) return 0;
  const int P = g.n / 32;
  return (P >= 2 && P <= 32 && (P & (P - 1)) == 0) ? P : 0;
}

cudaError_t pipe_upload_constants() { return upload_w96(); }

// One DST pass of the FP32 apply; B.pipe_pd is the common P of every instance.
cudaError_t pipe_dst_pass(const Batch& B, int axis, int in_slot, int out_slot) {
  switch (B.pipe_pd) {
    case 2: return dst_pass_p<2>(B, axis, in_slot, out_slot);
    case 4: return dst_pass_p<4>(B, axis, in_slot, out_slot);
    case 8: return dst_pass_p<8>(B, axis, in_slot, out_slot);
    case 16: return dst_pass_p<16>(B, axis, in_slot, out_slot);
    case 32: return dst_pass_p<32>(B, axis, in_slot, out_slot);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t pipe_time_pass(const Batch& B, int kind) {
  switch (B.pipe_pt) {
    case 2: return launch_time<2>(B, kind);
    case 4: return launch_time<4>(B, kind);
    case 8: return launch_time<8>(B, kind);
    case 16: return launch_time<16>(B, kind);
    case 32: return launch_time<32>(B, kind);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pcb
