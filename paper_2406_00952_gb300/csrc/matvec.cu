// All-at-once operator products (paper Sec. 1, Eqs. matrix_A, matrix_A_hat, matrix_T):
//     A     [x1; x2] = [alpha x1 + T^T x2 ; T x1 - alpha x2]
//     A_hat [x1; x2] = [T x1 - alpha x2 ; alpha x1 + T^T x2]
//     T = B_n (x) I + tau I (x) K,  B_n = B^(1) (B^(2))^{-1}.
// B_n x is applied per spatial column as the bidiagonal recurrence z_t = (x_t - (1-theta) z_{t-1})/theta
// followed by z_t - z_{t-1}; B_n^T x marches backward.  For theta = 1 (B_n = B^(1)) there is no
// recurrence and one fused pass over (t, x) reads x once and writes both output halves.
// K is the 5-point stencil (constant a: a (4u - sum of neighbours)/h^2; variable a: conservative
// edge-weighted form).  A neighbour outside the grid is 0 (Dirichlet) or the mirror image of the
// neighbour across the node (Neumann, Example 3: u_{-1} = u_1, u_N = u_{N-2}).  Epilogues fuse the
// Krylov updates that consume the product.
#include "pcb_internal.cuh"

namespace pcb {

enum { EPI_PLAIN = 0, EPI_RESID = 1, EPI_MINRES = 2 };
// flag on the epilogue kind: the product of an inner MINRES iteration of a mixed-precision solve,
// in two-word FP32 arithmetic where the instance allows it (k_matvec_tw)
constexpr int EPI_FAST = 8;

// tau*K u at spatial point (i, j) of the time block `u`
__device__ __forceinline__ double tauK(const Geom& g, const double* __restrict__ u, int i, int j, int col) {
  const int N = g.N;
  const double uc = u[col];
  double l, r, d, t;
  if (g.bc == PCB_BC_NEUMANN) {      // N >= 3: the mirrored neighbour always exists
    l = u[i > 0 ? col - 1 : col + 1];
    r = u[i < N - 1 ? col + 1 : col - 1];
    d = u[j > 0 ? col - N : col + N];
    t = u[j < N - 1 ? col + N : col - N];
  } else {
    l = i > 0 ? u[col - 1] : 0.0;
    r = i < N - 1 ? u[col + 1] : 0.0;
    d = j > 0 ? u[col - N] : 0.0;
    t = j < N - 1 ? u[col + N] : 0.0;
  }
  if (!g.var_a) {
    const double s = (l + r) + (d + t);
    return fma(-g.c, s, 4.0 * g.c * uc);
  }
  const double* ax = g.axs + (long long)j * (N + 1);
  const double* ay = g.ays;
  double s = ax[i] * l;
  s = fma(ax[i + 1], r, s);
  s = fma(ay[(long long)j * N + i], d, s);
  s = fma(ay[(long long)(j + 1) * N + i], t, s);
  return fma(g.dgs[col], uc, -s);
}

__device__ __forceinline__ void block_reduce_store(double v, double* dst) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) *dst = v;
  }
}

// Epilogue for one output value `o` = (op x)[idx]:
//   PLAIN : out = o
//   RESID : out = b - o,            partial += out^2
//   MINRES: out = o/beta - (beta/oldb) r1 (itn >= 2), partial += x*out/beta   (x is the Lanczos y)
struct Epi {
  int kind;
  double s, c;       // out = s*o + c*aux  (MINRES) ; for RESID s = -1, c = 1 (aux = b)
  double ds;         // dot scale
};

__device__ __forceinline__ double epi_apply(const Epi& e, double o, const double* __restrict__ aux,
                                            const double* __restrict__ xv, long long idx, double& part) {
  if (e.kind == EPI_PLAIN) return o;
  if (e.kind == EPI_RESID) {
    const double v = aux[idx] - o;
    part = fma(v, v, part);
    return v;
  }
  double v = e.s * o;
  if (e.c != 0.0) v = fma(e.c, aux[idx], v);
  part = fma(xv[idx], v, part);
  return v;
}

__device__ __forceinline__ Epi make_epi(int kind, const Scal* sc) {
  Epi e; e.kind = kind; e.s = 1.0; e.c = 0.0; e.ds = 1.0;
  if (kind == EPI_MINRES) {
    e.s = 1.0 / sc->beta;
    e.c = sc->itn >= 1 ? -(sc->beta / sc->oldb) : 0.0;
  }
  return e;
}

// Blocks of kMvThreads threads, one spatial column per thread.  theta == 1: blocks =
// ceil(m/kMvThreads) * ceil(n/tchunk) (fused); else blocks = 2 * ceil(m/kMvThreads) (forward-marching
// T role, backward-marching T^T role), each thread marching over all n time steps.  The marching
// form has only 2m threads, so the block is small enough that they all fit on the device at once:
// with 256-thread blocks a problem of m = 66,049 columns needed a second wave of 62 blocks, which
// took as long as the first.
constexpr int kMvThreads = 128;
__host__ __device__ int tw_patches(int N);
static_assert(32 * 4 == kMvThreads, "two-word product: one thread per point of a 32 x 4 patch");

void matvec_shape(Geom& g) {
  const int ncb = (g.m + kMvThreads - 1) / kMvThreads;
  if (g.theta == 1.0) {
    // time chunks: enough blocks of 256 threads' worth of columns to fill the device 16 times over
    const long long ncb256 = (g.m + 255) / 256;
    const int tch = (int)std::min<long long>(32, std::max<long long>(1, (ncb256 * g.n) / 2432));
    g.mv_tchunk = tch;
    // the two-word product (constant coefficient) tiles the grid in patches of its own
    const int units = g.var_a ? ncb : std::max(ncb, tw_patches(g.N));
    g.mv_blocks = units * ((g.n + tch - 1) / tch);
  } else {
    g.mv_tchunk = g.n;
    g.mv_blocks = 2 * ncb;
  }
}

// The FP64 product of block lb of one instance with its epilogue; returns the block's epilogue
// partial (for MINRES already scaled by 1/beta, as the scalar step expects).
__device__ __forceinline__ double matvec_block(const Geom& g, int lb, int op, const double* __restrict__ x,
                                               double* __restrict__ out, const double* __restrict__ aux,
                                               const Epi& e, int epi_kind) {
  const int N = g.N, m = g.m, n = g.n;
  const long long mn = g.mn;
  const double* __restrict__ x1 = x;
  const double* __restrict__ x2 = x + mn;
  // output half of the T x1 - alpha x2 rows and of the alpha x1 + T^T x2 rows
  const long long offT = (op == PCB_OP_A) ? mn : 0;
  const long long offTT = (op == PCB_OP_A) ? 0 : mn;
  const int ncb = (m + kMvThreads - 1) / kMvThreads;
  const double alpha = g.alpha;
  double part = 0.0;

  if (g.theta == 1.0 && !g.var_a && epi_kind != EPI_PLAIN) {
    // Same product with the epilogue's scale folded into the operator's coefficients (the kernel
    // is bound by FP64 instruction issue): out = sg*o + kp*aux with
    //   sg*(T x1 - alpha x2)   = (sg x1_t - sg x1_{t-1}) + (sg c)(4 u - sum of neighbours) - (sg alpha) x2
    //   sg*(alpha x1 + T^T x2) = (sg x2_t - sg x2_{t+1}) + (sg c)(4 u - sum of neighbours) + (sg alpha) x1
    // (MINRES: sg = 1/beta, kp = -beta/oldb; residual: sg = -1, kp = 1): ten FP64 operations per
    // output value instead of eleven.  The inner iterations of a mixed-precision solve use the
    // two-word FP32 form of this product instead (k_matvec_tw).
    const double sg = epi_kind == EPI_MINRES ? e.s : -1.0;
    const double kp = epi_kind == EPI_MINRES ? e.c : 1.0;
    const double sgc = sg * g.c, sga = sg * alpha;
    const int cb = lb % ncb, tc = lb / ncb;
    const int col = cb * kMvThreads + threadIdx.x;
    // an instance may have more blocks than this layout uses (the two-word layout's count)
    if (col < m && tc * g.mv_tchunk < n) {
      const int j = col / N, i = col - j * N;
      // neighbour offsets; at a Neumann boundary the missing one is the mirrored neighbour, at a
      // Dirichlet boundary it is masked to zero below
      const bool neu = g.bc == PCB_BC_NEUMANN;
      const int oL = i > 0 ? -1 : (neu ? 1 : 0), oR = i < N - 1 ? 1 : (neu ? -1 : 0);
      const int oD = j > 0 ? -N : (neu ? N : 0), oU = j < N - 1 ? N : (neu ? -N : 0);
      const bool zL = oL == 0, zR = oR == 0, zD = oD == 0, zU = oU == 0;
      const int t0 = tc * g.mv_tchunk;
      const int t1 = min(n, t0 + g.mv_tchunk);
      double x1p = t0 > 0 ? x1[(long long)(t0 - 1) * m + col] : 0.0;
      double x2c = x2[(long long)t0 * m + col];
      double s1p = sg * x1p, s2c = sg * x2c;     // scaled values carried by the ten-operation form
      for (int t = t0; t < t1; ++t) {
        const long long a = (long long)t * m + col;
        const double* u1 = x1 + (long long)t * m;
        const double* u2 = x2 + (long long)t * m;
        const double x1c = u1[col];
        const double x2n = t + 1 < n ? x2[a + m] : 0.0;
        const double nb1 = ((zL ? 0.0 : u1[col + oL]) + (zR ? 0.0 : u1[col + oR])) +
                           ((zD ? 0.0 : u1[col + oD]) + (zU ? 0.0 : u1[col + oU]));
        const double nb2 = ((zL ? 0.0 : u2[col + oL]) + (zR ? 0.0 : u2[col + oR])) +
                           ((zD ? 0.0 : u2[col + oD]) + (zU ? 0.0 : u2[col + oU]));
        const double s1 = sg * x1c, s2n = sg * x2n;
        double vT = fma(-sga, x2c, s1 - s1p);
        vT = fma(sgc, fma(4.0, x1c, -nb1), vT);
        double vTT = fma(sga, x1c, s2c - s2n);
        vTT = fma(sgc, fma(4.0, x2c, -nb2), vTT);
        s1p = s1;
        s2c = s2n;
        if (kp != 0.0) {
          vT = fma(kp, aux[offT + a], vT);
          vTT = fma(kp, aux[offTT + a], vTT);
        }
        if (epi_kind == EPI_MINRES) {
          part = fma(x[offT + a], vT, part);
          part = fma(x[offTT + a], vTT, part);
        } else {
          part = fma(vT, vT, part);
          part = fma(vTT, vTT, part);
        }
        out[offT + a] = vT;
        out[offTT + a] = vTT;
        x1p = x1c;
        x2c = x2n;
      }
    }
  } else if (g.theta == 1.0) {
    const int cb = lb % ncb, tc = lb / ncb;
    const int col = cb * kMvThreads + threadIdx.x;
    if (col < m && tc * g.mv_tchunk < n) {
      const int j = col / N, i = col - j * N;
      const int t0 = tc * g.mv_tchunk;
      const int t1 = min(n, t0 + g.mv_tchunk);
      const double d1 = 1.0;   // B^(1) diagonal
      double x1prev = t0 > 0 ? x1[(long long)(t0 - 1) * m + col] : 0.0;
      for (int t = t0; t < t1; ++t) {
        const long long a = (long long)t * m + col;
        const double* u1 = x1 + (long long)t * m;
        const double* u2 = x2 + (long long)t * m;
        const double x1c = u1[col], x2c = u2[col];
        const double x2n = t + 1 < n ? x2[a + m] : 0.0;
        // T x1 - alpha x2 = (x1c - x1prev) + tauK x1 - alpha x2
        double oT = fma(d1, x1c, -x1prev) + tauK(g, u1, i, j, col);
        oT = fma(-alpha, x2c, oT);
        // alpha x1 + T^T x2 = alpha x1 + (x2c - x2n) + tauK x2
        double oTT = (x2c - x2n) + tauK(g, u2, i, j, col);
        oTT = fma(alpha, x1c, oTT);
        out[offT + a] = epi_apply(e, oT, aux, x, offT + a, part);
        out[offTT + a] = epi_apply(e, oTT, aux, x, offTT + a, part);
        x1prev = x1c;
      }
    }
  } else {
    const int role = lb / ncb, cb = lb - role * ncb;
    const int col = cb * kMvThreads + threadIdx.x;
    if (col < m) {
      const int j = col / N, i = col - j * N;
      const double th = g.theta, om = 1.0 - th, ith = 1.0 / th;
      if (role == 0) {
        // forward: z_t = (x1_t - (1-theta) z_{t-1})/theta, (B_n x1)_t = z_t - z_{t-1}
        double zprev = 0.0;
#pragma unroll 2
        for (int t = 0; t < n; ++t) {
          const long long a = (long long)t * m + col;
          const double* u1 = x1 + (long long)t * m;
          const double z = fma(-om, zprev, u1[col]) * ith;
          double oT = (z - zprev) + tauK(g, u1, i, j, col);
          oT = fma(-alpha, x2[a], oT);
          out[offT + a] = epi_apply(e, oT, aux, x, offT + a, part);
          zprev = z;
        }
      } else {
        // backward: u_t = (x2_t - (1-theta) u_{t+1})/theta, (B_n^T x2)_t = u_t - u_{t+1}
        double unext = 0.0;
#pragma unroll 2
        for (int t = n - 1; t >= 0; --t) {
          const long long a = (long long)t * m + col;
          const double* u2 = x2 + (long long)t * m;
          const double u = fma(-om, unext, u2[col]) * ith;
          double oTT = (u - unext) + tauK(g, u2, i, j, col);
          oTT = fma(alpha, x1[a], oTT);
          out[offTT + a] = epi_apply(e, oTT, aux, x, offTT + a, part);
          unext = u;
        }
      }
    }
  }
  if (epi_kind == EPI_MINRES) part *= e.s;
  return part;
}

__global__ void __launch_bounds__(kMvThreads) k_matvec(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                const int* __restrict__ active, int op, int x_slot, int out_slot,
                                                int aux_slot, int epi_kind, double* __restrict__ partial) {
  const int inst = find_inst(off, count, blockIdx.x);
  if (active && !active[inst]) return;
  const Geom& g = G[inst];
  const double* __restrict__ aux = aux_slot >= 0 ? S[inst].v[aux_slot] : nullptr;
  const double part = matvec_block(g, blockIdx.x - off[inst], op, S[inst].v[x_slot], S[inst].v[out_slot], aux,
                                   make_epi(epi_kind, Sc + inst), epi_kind);
  if (partial && epi_kind != EPI_PLAIN) block_reduce_store(part, partial + blockIdx.x);
}

// ------------------------------------------------------------------------------------------
// Two-word FP32 product for the inner iterations of a mixed-precision MINRES solve (theta = 1,
// constant coefficient, Lanczos epilogue):
//     out = A y / beta - (beta/oldb) r1,   partial = y . out / beta   (A: Eq. matrix_A)
// On this GPU FP64 instructions issue at 1/64 of the FP32 rate, and the FP64 form above is
// bound by them (ten per output value).  Here every FP64 input is split, with integer
// operations, into two FP32 words that hold the leading 24 and the next 23 bits of its
// significand (47 of its 53 bits), and the product is evaluated in two-word arithmetic built
// from error-free transformations: Knuth's two-sum, Dekker's fast two-sum and the FMA-based
// exact product (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2), on packed pairs of FP32 lanes that
// carry the two output rows of a point (T x1 - alpha x2 and alpha x1 + T^T x2) side by side.
// Each result is accurate to about 2^-46 of the magnitudes of its terms (the FP64 form: 2^-53),
// which the iteration does not notice next to the FP32 preconditioner's rounding.  Results are
// widened to FP64 with integer operations and one FP64 add per value.
//
// Scaling: y is split as y 2^-ky and r1 as r1 2^-ka, with 2^ky and 2^ka the binades of beta and
// oldb, so the words stay far inside the FP32 range whatever the scale of the right-hand side
// (the coefficients absorb 2^ky and 2^ka exactly).  A scaled value below 2^-103 becomes 0 (an
// absolute error far below the rest); one beyond the FP32 range becomes NaN, which the
// iteration's non-finite check reports.
//
// Layout: a block of 128 threads owns a patch of 32 x 4 spatial points (x1 fastest) and a chunk
// of time levels.  For each level t the split words of x1(t) and x2(t) on the patch and its
// one-point halo (Dirichlet: zero outside the grid; Neumann: the mirrored neighbour) sit in a
// shared-memory tile of (x1 hi, x2 hi, x1 lo, x2 lo); three tiles rotate (t, t+1 being read,
// t+2 being filled from loads issued one step ahead).
// ------------------------------------------------------------------------------------------
namespace tw {

constexpr int kI = 32, kJ = 4;                  // patch: x1 by x2 points (kI * kJ = kMvThreads)
constexpr int kW = kI + 2, kH = kJ + 2;         // with the halo
constexpr int kSlots = kW * kH;
constexpr int kHalo = 2 * kI + 2 * kJ;          // halo points (corners unused)

using f2 = float2;
__device__ __forceinline__ f2 pk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 sub(f2 a, f2 b) { return __ffma2_rn(make_float2(-1.f, -1.f), b, a); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 swp(f2 a) { return make_float2(a.y, a.x); }

// s + e = a + b exactly (two-sum)
__device__ __forceinline__ void two_sum(f2 a, f2 b, f2& s, f2& e) {
  s = add(a, b);
  const f2 bb = sub(s, a);
  e = add(sub(a, sub(s, bb)), sub(b, bb));
}
// s + e = a - b exactly
__device__ __forceinline__ void two_diff(f2 a, f2 b, f2& s, f2& e) {
  s = sub(a, b);
  const f2 bb = sub(s, a);
  e = sub(sub(a, sub(s, bb)), add(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (fast two-sum); renormalises a word pair
__device__ __forceinline__ void renorm(f2& a, f2& b) {
  const f2 s = add(a, b);
  b = sub(b, sub(s, a));
  a = s;
}
// (ph, pl) ~ k * (xh + xl) for a two-word coefficient (kh, kl) with nkh = -kh: the leading
// product is exact in ph - nerr (nerr = ph - kh*xh exactly, by one FMA), the cross terms are
// rounded once each.
__device__ __forceinline__ void prod(f2 kh, f2 kl, f2 nkh, f2 xh, f2 xl, f2& ph, f2& pl) {
  ph = mul(kh, xh);
  const f2 nerr = fma2(nkh, xh, ph);
  pl = sub(fma2(kh, xl, mul(kl, xh)), nerr);
}
// (h, l) += (ph, pl), unnormalised
__device__ __forceinline__ void acc(f2& h, f2& l, f2 ph, f2 pl) {
  f2 s, e;
  two_sum(h, ph, s, e);
  h = s;
  l = add(l, add(e, pl));
}

// x 2^-k split into two FP32 words (b20 = (896 + k) << 20, the FP64 exponent bias of the scaled
// value): hi = the leading 24 bits of the significand, lo = the next 23 (both truncated), so
// |x 2^-k - hi - lo| < 2^-46 |x 2^-k|.  The second word is the difference of two FP32 numbers of
// the same binade (exact).  Scaled values below 2^-103 and FP64 subnormals become 0.
__device__ __forceinline__ void split(double x, int b20, float& hi, float& lo) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const unsigned sgn = hw & 0x80000000u;
  const int u = (int)(hw & 0x7fffffffu) - b20;             // FP32 exponent field at bit 20
  const unsigned hb = (__funnelshift_l(lw, (unsigned)u, 3) & 0x7fffffffu) | sgn;
  const unsigned s3 = ((unsigned)u << 3) - (23u << 23);     // unit of the second word
  const unsigned one = (s3 & 0x7f800000u) | sgn;
  const float l = __fsub_rn(__uint_as_float(one | ((lw >> 6) & 0x007fffffu)), __uint_as_float(one));
  // a normal FP64 value whose scaled exponent lies in [-103, 127] (zeros and FP64 subnormals give 0)
  const bool ok = (hw & 0x7ff00000u) != 0u && (unsigned)(u - (24 << 20)) < (231u << 20);
  hi = ok ? __uint_as_float(hb) : (u >= (255 << 20) ? __uint_as_float(0x7fc00000u) : 0.f);
  lo = ok ? l : 0.f;
}
// exact FP64 value of an FP32 word (subnormal words give 0; infinities and NaN are kept)
__device__ __forceinline__ double widen(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu;
  unsigned hw = (b & 0x80000000u) | ((a >> 3) + (896u << 20));
  if (a >= 0x7f800000u) hw |= 0x7ff00000u;
  const bool z = a < 0x00800000u;
  return __hiloint2double((int)(z ? (b & 0x80000000u) : hw), (int)(z ? 0u : (b << 29)));
}
// a second word (never infinite or NaN when its leading word is finite)
__device__ __forceinline__ double widen_lo(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7fffffffu;
  const bool z = a < 0x00800000u;
  const unsigned hw = (b & 0x80000000u) | ((a >> 3) + (896u << 20));
  return __hiloint2double((int)(z ? 0u : hw), (int)(z ? 0u : (b << 29)));
}
// binade exponent of a positive normal double (0 otherwise)
__device__ __forceinline__ int binade(double v) {
  const int e = (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu);
  return (v > 0.0 && e > 0 && e < 2047) ? e - 1023 : 0;
}
__device__ __forceinline__ double pow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }
__device__ __forceinline__ void split_rn(double v, float& h, float& l) {
  h = __double2float_rn(v);
  l = __double2float_rn(v - (double)h);
}

// grid column of tile point (gi, gj) in [-1, N] x [-1, N], or -1 for a zero
__device__ __forceinline__ int tile_src(int gi, int gj, int N, bool neu) {
  if (neu) {
    const bool oi = gi < 0 || gi >= N, oj = gj < 0 || gj >= N;
    if (oi && oj) return -1;
    if (gi == -1) gi = 1; else if (gi == N) gi = N - 2;
    if (gj == -1) gj = 1; else if (gj == N) gj = N - 2;
  }
  if (gi < 0 || gi >= N || gj < 0 || gj >= N) return -1;
  return gj * N + gi;
}

}  // namespace tw

__host__ __device__ int tw_patches(int N) { return ((N + tw::kI - 1) / tw::kI) * ((N + tw::kJ - 1) / tw::kJ); }

// Block lb of one instance (theta = 1, constant coefficient) of the two-word product with the
// MINRES epilogue e; returns the block's partial of y . out / beta.
__device__ __forceinline__ double matvec_tw_block(const Geom& g, int lb, int op, const double* __restrict__ x,
                                                  double* __restrict__ out, const double* __restrict__ aux,
                                                  const Epi& e, const Scal& sc, float4 (*tile)[tw::kSlots]) {
  using namespace tw;
  const int N = g.N, m = g.m, n = g.n;
  const long long mn = g.mn;
  const int npi = (N + kI - 1) / kI, npatch = tw_patches(N);
  const int p = lb % npatch, tc = lb / npatch;
  const int t0 = tc * g.mv_tchunk;
  if (t0 >= n) return 0.0;          // the FP64 layout of this instance may use more blocks
  const int t1 = min(n, t0 + g.mv_tchunk);
  const int i0 = (p % npi) * kI, j0 = (p / npi) * kJ;
  const int ti = threadIdx.x % kI, tj = threadIdx.x / kI;
  const int i = i0 + ti, j = j0 + tj;
  const bool own = i < N && j < N;
  const bool neu = g.bc == PCB_BC_NEUMANN;
  const int os = (tj + 1) * kW + ti + 1;           // this thread's point in the tile
  const int osrc = tile_src(i, j, N, neu);
  const int col = own ? osrc : 0;
  int hs = -1, hsrc = -1;                          // one halo point per thread below kHalo
  if (threadIdx.x < kHalo) {
    const int h = threadIdx.x;
    int r, q;
    if (h < kI) { r = 0; q = h + 1; }
    else if (h < 2 * kI) { r = kJ + 1; q = h - kI + 1; }
    else if (h < 2 * kI + kJ) { r = h - 2 * kI + 1; q = 0; }
    else { r = h - 2 * kI - kJ + 1; q = kI + 1; }
    hs = r * kW + q;
    hsrc = tile_src(i0 + q - 1, j0 + r - 1, N, neu);
  }
  // scalings (powers of two) and two-word coefficients
  const int ky = binade(sc.beta);
  const bool use_aux = e.c != 0.0;
  const int ka = use_aux ? binade(sc.oldb) : 0;
  const double sgd = e.s * pow2(ky), kpd = e.c * pow2(ka);
  const int by = (896 + ky) * (1 << 20), ba = (896 + ka) * (1 << 20);
  float w0, w1;
  split_rn(sgd, w0, w1);
  const f2 SGh = pk(w0, w0), SGl = pk(w1, w1), nSG = pk(-w0, -w0);
  split_rn(g.c, w0, w1);
  const f2 Ch = pk(w0, w0), Cl = pk(w1, w1), nC = pk(-w0, -w0);
  split_rn(g.alpha, w0, w1);
  const f2 ALh = pk(-w0, w0), ALl = pk(-w1, w1), nAL = pk(w0, -w0);   // -alpha x2 | +alpha x1
  split_rn(kpd, w0, w1);
  const f2 KPh = pk(w0, w0), KPl = pk(w1, w1), nKP = pk(-w0, -w0);
  const long long offT = (op == PCB_OP_A) ? mn : 0;
  const long long offTT = (op == PCB_OP_A) ? 0 : mn;

  // raw loads of tile tt (own point and halo point, both halves) and their split into the tile
  auto fetch = [&](int tt, double& a1, double& a2, double& h1, double& h2) {
    const long long base = (long long)tt * m;
    const bool in = tt < n;
    a1 = (in && osrc >= 0) ? x[base + osrc] : 0.0;
    a2 = (in && osrc >= 0) ? x[mn + base + osrc] : 0.0;
    h1 = (in && hsrc >= 0) ? x[base + hsrc] : 0.0;
    h2 = (in && hsrc >= 0) ? x[mn + base + hsrc] : 0.0;
  };
  auto store = [&](int b, double a1, double a2, double h1, double h2) {
    float4 v;
    split(a1, by, v.x, v.z);
    split(a2, by, v.y, v.w);
    tile[b][os] = v;
    if (hs >= 0) {
      split(h1, by, v.x, v.z);
      split(h2, by, v.y, v.w);
      tile[b][hs] = v;
    }
  };
  {
    double a1, a2, h1, h2;
    fetch(t0, a1, a2, h1, h2);
    store(0, a1, a2, h1, h2);
    fetch(t0 + 1, a1, a2, h1, h2);
    store(1, a1, a2, h1, h2);
  }
  float x1ph = 0.f, x1pl = 0.f;                    // x1(t-1) at this point
  if (own && t0 > 0) split(x[(long long)(t0 - 1) * m + col], by, x1ph, x1pl);
  double ra = 0.0, rb = 0.0;                       // r1 at (t, point), both halves
  if (own && use_aux) { ra = aux[offT + (long long)t0 * m + col]; rb = aux[offTT + (long long)t0 * m + col]; }
  f2 dh = pk(0.f, 0.f), dl = pk(0.f, 0.f);         // y . out (scaled), two words per lane
  __syncthreads();
  int b0 = 0, b1 = 1, b2 = 2;                      // tiles of levels t, t+1, t+2
  for (int t = t0; t < t1; ++t) {
    const bool pre = t + 2 <= t1;                  // level t+2 is read by step t+1
    double n1 = 0.0, n2 = 0.0, nh1 = 0.0, nh2 = 0.0, nra = 0.0, nrb = 0.0;
    if (pre) fetch(t + 2, n1, n2, nh1, nh2);
    if (own && use_aux && t + 1 < t1) {
      nra = aux[offT + (long long)(t + 1) * m + col];
      nrb = aux[offTT + (long long)(t + 1) * m + col];
    }
    if (own) {
      const float4 c = tile[b0][os];
      const float4 qL = tile[b0][os - 1], qR = tile[b0][os + 1], qD = tile[b0][os - kW], qU = tile[b0][os + kW];
      const float4 q1 = tile[b1][os];
      const f2 ch = pk(c.x, c.y), cl = pk(c.z, c.w);
      // (x1(t) - x1(t-1) | x2(t) - x2(t+1))
      f2 H, L, ex;
      two_diff(ch, pk(x1ph, q1.y), H, ex);
      L = add(sub(cl, pk(x1pl, q1.w)), ex);
      // 4 u - (sum of the four neighbours), renormalised before it is scaled
      f2 lh, ll;
      {
        f2 s1, e1, s2, e2, s, e3;
        two_sum(pk(qL.x, qL.y), pk(qR.x, qR.y), s1, e1);
        two_sum(pk(qD.x, qD.y), pk(qU.x, qU.y), s2, e2);
        two_sum(s1, s2, s, e3);
        const f2 sl = add(add(add(pk(qL.z, qL.w), pk(qR.z, qR.w)), add(pk(qD.z, qD.w), pk(qU.z, qU.w))),
                          add(add(e1, e2), e3));
        const f2 four = pk(4.f, 4.f);
        two_diff(mul(four, ch), s, lh, ex);
        ll = sub(fma2(four, cl, ex), sl);
        renorm(lh, ll);
      }
      f2 ph, pl;
      prod(Ch, Cl, nC, lh, ll, ph, pl);              // + c (4 u - sum)
      acc(H, L, ph, pl);
      prod(ALh, ALl, nAL, swp(ch), swp(cl), ph, pl); // - alpha x2 | + alpha x1
      acc(H, L, ph, pl);
      renorm(H, L);
      f2 oh, ol;
      prod(SGh, SGl, nSG, H, L, oh, ol);             // 2^ky / beta
      if (use_aux) {
        float rah, ral, rbh, rbl;
        split(ra, ba, rah, ral);
        split(rb, ba, rbh, rbl);
        prod(KPh, KPl, nKP, pk(rah, rbh), pk(ral, rbl), ph, pl);   // - (beta/oldb) r1
        acc(oh, ol, ph, pl);
      }
      renorm(oh, ol);
      const long long a = (long long)t * m + col;
      out[offT + a] = widen(oh.x) + widen_lo(ol.x);
      out[offTT + a] = widen(oh.y) + widen_lo(ol.y);
      // epilogue: y at each output's own index times the output
      const f2 yh = (op == PCB_OP_A) ? swp(ch) : ch, yl = (op == PCB_OP_A) ? swp(cl) : cl;
      prod(yh, yl, mul(yh, pk(-1.f, -1.f)), oh, ol, ph, pl);
      acc(dh, dl, ph, pl);
      x1ph = c.x;
      x1pl = c.z;
    }
    if (pre) store(b2, n1, n2, nh1, nh2);
    ra = nra;
    rb = nrb;
    __syncthreads();
    const int bt = b0;
    b0 = b1; b1 = b2; b2 = bt;
  }
  if (!own) return 0.0;
  // y . out / beta = (2^ky / beta) * sum of (y 2^-ky) . out
  return ((widen(dh.x) + widen(dh.y)) + (widen(dl.x) + widen(dl.y))) * sgd;
}

__global__ void __launch_bounds__(kMvThreads) k_matvec_tw(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                   Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                   const int* __restrict__ active, int op, int x_slot, int out_slot,
                                                   int aux_slot, double* __restrict__ partial) {
  __shared__ float4 tile[3][tw::kSlots];
  const int inst = find_inst(off, count, blockIdx.x);
  if (active && !active[inst]) return;
  const Geom& g = G[inst];
  const double* __restrict__ aux = aux_slot >= 0 ? S[inst].v[aux_slot] : nullptr;
  const Epi e = make_epi(EPI_MINRES, Sc + inst);
  const int lb = blockIdx.x - off[inst];
  const double part = (g.theta == 1.0 && !g.var_a)
                          ? matvec_tw_block(g, lb, op, S[inst].v[x_slot], S[inst].v[out_slot], aux, e, Sc[inst], tile)
                          : matvec_block(g, lb, op, S[inst].v[x_slot], S[inst].v[out_slot], aux, e, EPI_MINRES);
  if (partial) block_reduce_store(part, partial + blockIdx.x);
}

// Epilogue of a finite-element product already written to out (see k_matvec's epilogues): one
// instance, grid-stride blocks, one partial per block (the layout the scalar steps read).
__global__ void __launch_bounds__(256) k_fem_epilogue(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                      Scal* __restrict__ Sc, int x_slot, int out_slot, int aux_slot,
                                                      int epi_kind, double* __restrict__ partial) {
  const Geom& g = G[0];
  const double* __restrict__ x = S[0].v[x_slot];
  double* __restrict__ out = S[0].v[out_slot];
  const double* __restrict__ aux = aux_slot >= 0 ? S[0].v[aux_slot] : nullptr;
  const Epi e = make_epi(epi_kind, Sc);
  const long long len = 2 * g.mn;
  double part = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    out[i] = epi_apply(e, out[i], aux, x, i, part);
  if (partial) {
    if (epi_kind == EPI_MINRES) part *= e.s;
    block_reduce_store(part, partial + blockIdx.x);
  }
}

cudaError_t launch_fem_spatial(const Batch& B, int mode, int op, int in_slot, int out_slot);

cudaError_t launch_matvec(const Batch& B, int op, int x_slot, int out_slot, int aux_slot, int epi) {
  if (B.fem_m > 0) {
    // finite elements: the product through the sine basis (FEM_PRODUCT = 2), then the epilogue
    cudaError_t e = launch_fem_spatial(B, 2, op, x_slot, out_slot);
    if (e != cudaSuccess || (epi & (EPI_FAST - 1)) == EPI_PLAIN) return e;
    k_fem_epilogue<<<B.tot_mv, 256, 0, B.stream>>>(B.G, B.S, B.Sc, x_slot, out_slot, aux_slot, epi & (EPI_FAST - 1),
                                                   B.partial);
    return cudaGetLastError();
  }
  if ((epi & EPI_FAST) && (epi & (EPI_FAST - 1)) == EPI_MINRES) {
    k_matvec_tw<<<B.tot_mv, kMvThreads, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_mv, B.count, B.active, op, x_slot,
                                                       out_slot, aux_slot, B.partial);
    return cudaGetLastError();
  }
  k_matvec<<<B.tot_mv, kMvThreads, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_mv, B.count, B.active, op, x_slot, out_slot,
                                           aux_slot, epi & (EPI_FAST - 1), B.partial);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// Right-hand side (Sec. 1: f~, g~ with M = I, then [g; sqrt(gamma) f] or [sqrt(gamma) f; g]).
// g, f: (n+1)*m samples; y0: m values or null.  One thread per (t, col).
// ------------------------------------------------------------------------------------------
__global__ void k_rhs(Geom g, int op, const double* __restrict__ gs, const double* __restrict__ fs,
                      const double* __restrict__ y0, double* __restrict__ b) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.mn) return;
  const int m = g.m, N = g.N;
  const int t = (int)(idx / m), col = (int)(idx - (long long)t * m);
  const double th = g.theta, tau = g.tau;
  double ft = tau * (th * fs[idx + m] + (1.0 - th) * fs[idx]);
  double gt = tau * (th * gs[idx] + (1.0 - th) * gs[idx + m]);
  if (t == 0 && y0) {
    const int j = col / N, i = col - j * N;
    const double Ky0 = tauK(g, y0, i, j, col) / tau;
    ft += y0[col] - (1.0 - th) * tau * Ky0;
    gt -= tau * (1.0 - th) * y0[col];
  }
  const double sf = g.sqrt_gamma * ft;
  if (op == PCB_OP_A) { b[idx] = gt; b[g.mn + idx] = sf; }
  else { b[idx] = sf; b[g.mn + idx] = gt; }
}

// y = (B2^{-1} (x) I) x1 / sqrt(gamma), p = (B2^{-T} (x) I) x2; one thread per column and half.
__global__ void k_recover(Geom g, const double* __restrict__ x, double* __restrict__ y, double* __restrict__ p) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = g.m, n = g.n;
  if (tid >= 2 * m) return;
  const int half = tid / m, col = tid - half * m;
  const double th = g.theta, om = 1.0 - th, ith = 1.0 / th;
  if (half == 0) {
    const double s = 1.0 / g.sqrt_gamma;
    double z = 0.0;
    for (int t = 0; t < n; ++t) {
      const long long a = (long long)t * m + col;
      z = fma(-om, z, x[a]) * ith;
      y[a] = z * s;
    }
  } else {
    double u = 0.0;
    for (int t = n - 1; t >= 0; --t) {
      const long long a = (long long)t * m + col;
      u = fma(-om, u, x[g.mn + a]) * ith;
      p[a] = u;
    }
  }
}

cudaError_t launch_rhs(const Geom& g, cudaStream_t st, int op, const double* gs, const double* fs, const double* y0,
                       double* b) {
  const long long blocks = (g.mn + 255) / 256;
  k_rhs<<<(unsigned)blocks, 256, 0, st>>>(g, op, gs, fs, y0, b);
  return cudaGetLastError();
}

// dst[0..n) = src[0..n) where one side is memory the device maps directly (page-locked host memory
// over the coherent CPU-GPU link): SM loads and stores instead of a copy-engine transfer, which on
// this system ran at 200 GB/s only some of the time (30-40 GB/s right after long kernel phases);
// 16-byte accesses when both pointers are 16-byte aligned.
__global__ void k_copy_mapped(const double* __restrict__ src, double* __restrict__ dst, long long n, int vec2) {
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long st = (long long)gridDim.x * blockDim.x;
  if (vec2) {
    // four 16-byte loads in flight per thread before their stores: reads of page-locked host
    // memory cross the CPU-GPU link with a long latency
    const double2* s2 = (const double2*)src;
    double2* d2 = (double2*)dst;
    const long long n2 = n / 2;
    long long i = i0;
    for (; i + 3 * st < n2; i += 4 * st) {
      const double2 a = s2[i], b = s2[i + st], c = s2[i + 2 * st], d = s2[i + 3 * st];
      d2[i] = a; d2[i + st] = b; d2[i + 2 * st] = c; d2[i + 3 * st] = d;
    }
    for (; i < n2; i += st) d2[i] = s2[i];
    if (i0 == 0 && (n & 1)) dst[n - 1] = src[n - 1];
  } else {
    for (long long i = i0; i < n; i += st) dst[i] = src[i];
  }
}

cudaError_t launch_copy_mapped(cudaStream_t st, const double* src, double* dst, long long n) {
  const int vec2 = (((uintptr_t)src | (uintptr_t)dst) & 15) == 0;
  k_copy_mapped<<<152 * 8, 256, 0, st>>>(src, dst, n, vec2);
  return cudaGetLastError();
}

cudaError_t launch_recover(const Geom& g, cudaStream_t st, const double* x, double* y, double* p) {
  const int blocks = (2 * g.m + 127) / 128;
  k_recover<<<blocks, 128, 0, st>>>(g, x, y, p);
  return cudaGetLastError();
}

}  // namespace pcb
