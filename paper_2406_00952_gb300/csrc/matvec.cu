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
// flag on the epilogue kind: the inner product of a mixed-precision MINRES iteration may use the
// nine-operation arithmetic of the theta = 1 product (see k_matvec)
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

void matvec_shape(Geom& g) {
  const int ncb = (g.m + kMvThreads - 1) / kMvThreads;
  if (g.theta == 1.0) {
    // time chunks: enough blocks of 256 threads' worth of columns to fill the device 16 times over
    const long long ncb256 = (g.m + 255) / 256;
    const int tch = (int)std::min<long long>(32, std::max<long long>(1, (ncb256 * g.n) / 2432));
    g.mv_tchunk = tch;
    g.mv_blocks = ncb * ((g.n + tch - 1) / tch);
  } else {
    g.mv_tchunk = g.n;
    g.mv_blocks = 2 * ncb;
  }
}

__global__ void __launch_bounds__(kMvThreads) k_matvec(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                Scal* __restrict__ Sc, const int* __restrict__ off, int count,
                                                const int* __restrict__ active, int op, int x_slot, int out_slot,
                                                int aux_slot, int epi_kind, double* __restrict__ partial) {
  const bool fast = (epi_kind & EPI_FAST) != 0;
  epi_kind &= EPI_FAST - 1;
  const int inst = find_inst(off, count, blockIdx.x);
  if (active && !active[inst]) return;
  const Geom& g = G[inst];
  const int lb = blockIdx.x - off[inst];
  const double* __restrict__ x = S[inst].v[x_slot];
  double* __restrict__ out = S[inst].v[out_slot];
  const double* __restrict__ aux = aux_slot >= 0 ? S[inst].v[aux_slot] : nullptr;
  const Epi e = make_epi(epi_kind, Sc + inst);
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
    // output value instead of eleven.  With EPI_FAST (the inner product of a mixed-precision
    // MINRES iteration) the time-difference and Laplacian diagonal terms share one coefficient,
    //   (sg + 4 sg c) u_t - sg u_{t-+1} -+ (sg alpha) x_other - (sg c)(sum of neighbours),
    // nine operations; on smooth vectors its rounding is about three times that of the ten-operation
    // form (the large diagonal term cancels against the neighbours last), which delays FP64 MINRES
    // at the bench size by two iterations but is far below the FP32 preconditioner's perturbation.
    const double sg = epi_kind == EPI_MINRES ? e.s : -1.0;
    const double kp = epi_kind == EPI_MINRES ? e.c : 1.0;
    const double sgc = sg * g.c, sga = sg * alpha, kd = fma(4.0, sgc, sg);
    const int cb = lb % ncb, tc = lb / ncb;
    const int col = cb * kMvThreads + threadIdx.x;
    if (col < m) {
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
        double vT, vTT;
        if (fast) {
          vT = fma(-sg, x1p, kd * x1c);
          vT = fma(-sga, x2c, vT);
          vT = fma(-sgc, nb1, vT);
          vTT = fma(-sg, x2n, kd * x2c);
          vTT = fma(sga, x1c, vTT);
          vTT = fma(-sgc, nb2, vTT);
        } else {
          const double s1 = sg * x1c, s2n = sg * x2n;
          vT = fma(-sga, x2c, s1 - s1p);
          vT = fma(sgc, fma(4.0, x1c, -nb1), vT);
          vTT = fma(sga, x1c, s2c - s2n);
          vTT = fma(sgc, fma(4.0, x2c, -nb2), vTT);
          s1p = s1;
          s2c = s2n;
        }
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
    if (col < m) {
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
  if (partial && epi_kind != EPI_PLAIN) {
    if (epi_kind == EPI_MINRES) part *= e.s;
    block_reduce_store(part, partial + blockIdx.x);
  }
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
  k_matvec<<<B.tot_mv, kMvThreads, 0, B.stream>>>(B.G, B.S, B.Sc, B.off_mv, B.count, B.active, op, x_slot, out_slot,
                                           aux_slot, epi, B.partial);
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
