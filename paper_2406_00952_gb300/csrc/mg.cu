// Multigrid preconditioner route for variable a(x) (paper Sec. 3.5, Step 2 by multigrid; Sec. 4).
//
// P_S^{-1} v: time DFT of both halves (zeta = pi scaling, packed as real/imaginary parts), then per
// frequency slot r the 2x2 block G = [[mu_r, -alpha], [alpha, conj(mu_r)]] is decoupled with
// Lemma 3.14 (G = W diag(D1, D2) W^{-1}, W = [[1, M], [M, 1]], D2 = conj(D1)); the two decoupled
// components are solved with `cycles` V-cycles on (D1 I + tau K) -- the second as the conjugate of
// a solve with a conjugated right-hand side -- then recoupled with W and transformed back.
// P_MS^{-1} v (Eq. matrix_P_MS): the same pipeline with no coupling and the real shift
// sigma_r = sqrt(|mu_r|^2 + alpha^2) for both halves.
// Only slots r < n/2 are solved: slot n-1-r carries the conjugate system, whose solution is the
// conjugate (this holds for any real-coefficient linear solver, the V-cycle included, because
// W_{n-1-r} equals conj(W_r) with its columns swapped up to scaling).
//
// V-cycle (reading of an unspecified method): vertex-centred coarsening N -> (N-1)/2, coarse edge
// coefficient = mean of the two fine edges it spans, full-weighting restriction, bilinear
// prolongation, damped Jacobi (weight 4/5), nu1 = nu2 = 2, exact solve on the 1 x 1 grid, zero
// initial guess; cycle c > 1 corrects with a V-cycle on the current residual.
// Neumann grids (Example 3 solved as in Sec. 4, constant a): N = 2^k + 1 nodes per side with the
// boundary, coarse nodes the even fine nodes, N -> (N+1)/2 down to 3; the mirrored stencil
// c (4u - sum of neighbours), c = tau a / h^2, on every level; full weighting with mirrored ghost
// values; bilinear prolongation; the same damped Jacobi; on the 3 x 3 grid an exact solve through
// the eigenvectors of the 3-node mirrored second difference.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fft_reg.cuh"

namespace pcb {

bool mg_available() { return true; }
int mg_launch_count(int kind);

static constexpr double kJacobiWeight = 0.8;
static constexpr int kMaxLevels = 12;
static constexpr int kNu = 2;
static long long g_mg_launches = 0;   // kernel launches issued by the multigrid route

struct MgLevel {
  int N;                      // interior points per side (Neumann: nodes per side with the boundary)
  int neu;                    // 1: Neumann grid, mirrored stencil with the constant c below
  double c; float cf;         // Neumann: tau a / h^2 of this level
  double* co;                 // Neumann coarsest level: [V2 (81) | V2^{-1} (81) | lambda (9)], FP64 ...
  float* cof;                 // ... and FP32
  double* axs;                // tau/h_l^2 * ax  (N x (N+1))
  double* ays;                // tau/h_l^2 * ay  ((N+1) x N)
  double* dgs;                // sum of the four  (N x N)
  float* axf; float* ayf; float* dgf;
  void* a[3];                 // work arrays: n systems x N^2 complex (FP64-sized)
};

struct MgHost {
  int nlev = 0;
  int nsys = 0;               // systems = n (n/2 frequency slots x 2 right-hand sides)
  int tail_l0 = -1;           // first level of the fused coarse-level launch (-1: none)
  MgLevel lev[kMaxLevels];
  void* zfine = nullptr;      // outer solution (level 0)
  void* xfine = nullptr;      // outer residual (level 0)
  double2* tab_d = nullptr;   // per slot r < n/2: {shift, coupling M, 1/(1-M^2)} for P_S, then P_MS shift
  float2* tab_f = nullptr;
};

// workspace registry: one MgHost per Geom (keyed by the workspace pointer)
static std::vector<std::pair<const void*, MgHost>>& registry() {
  static std::vector<std::pair<const void*, MgHost>> r;
  return r;
}
static MgHost* find_host(const void* ws) {
  for (auto& e : registry())
    if (e.first == ws) return &e.second;
  return nullptr;
}

static int levels_for(int N, bool neu = false) {
  int l = 1;
  if (neu) { while (N > 3) { N = (N + 1) / 2; ++l; } return l; }
  while (N > 1) { N = (N - 1) / 2; ++l; }
  return l;
}

size_t mg_workspace_bytes(const Geom& g) {
  size_t b = 0;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int N = g.N;
  const bool neu = g.bc == PCB_BC_NEUMANN;
  const size_t nsys = (size_t)g.n;
  for (int l = 0; l < levels_for(g.N, neu); ++l) {
    const size_t ne = (size_t)N * (N + 1), nn = (size_t)N * N;
    if (!neu) b += up(ne * 8) * 2 + up(nn * 8) + up(ne * 4) * 2 + up(nn * 4);
    b += 3 * up(nsys * nn * sizeof(double2));
    if (l == 0) b += 2 * up(nsys * nn * sizeof(double2));
    N = neu ? (N + 1) / 2 : (N - 1) / 2;
  }
  if (neu) b += up(171 * 8) + up(171 * 4);
  b += up((size_t)g.n * 3 * sizeof(double2)) + up((size_t)g.n * 3 * sizeof(float2));
  return b;
}

// Neumann levels: every level's c = tau a / h_l^2, work arrays, and on the 3 x 3 grid the exact
// solve's tables.  The 3-node mirrored second difference [[2,-2,0],[-1,2,-1],[0,-2,2]] has the
// eigenvalues 0, 2, 4 with eigenvectors (1,1,1), (1,0,-1), (1,-1,1); the 2D operator on the 3 x 3
// grid is c (D (x) I + I (x) D), diagonal in V (x) V.
static unsigned char* mg_setup_neumann(const Geom& g, MgHost& h, unsigned char* p, double a0) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int N = g.N;
  for (int l = 0; l < h.nlev; ++l) {
    MgLevel& L = h.lev[l];
    std::memset(&L, 0, sizeof(L));
    L.N = N; L.neu = 1;
    const double hl = 1.0 / (N - 1);
    L.c = g.tau * a0 / (hl * hl);
    L.cf = (float)L.c;
    const size_t nn = (size_t)N * N;
    for (int k = 0; k < 3; ++k) { L.a[k] = p; p += up((size_t)h.nsys * nn * sizeof(double2)); }
    if (l == 0) {
      h.zfine = p; p += up((size_t)h.nsys * nn * sizeof(double2));
      h.xfine = p; p += up((size_t)h.nsys * nn * sizeof(double2));
    }
    N = (N + 1) / 2;
  }
  MgLevel& C = h.lev[h.nlev - 1];
  const double V[3][3] = {{1, 1, 1}, {1, 0, -1}, {1, -1, 1}};          // columns: eigenvectors
  const double Vi[3][3] = {{0.25, 0.5, 0.25}, {0.5, 0.0, -0.5}, {0.25, -0.5, 0.25}};   // V^{-1}
  const double lam[3] = {0.0, 2.0, 4.0};
  std::vector<double> co(171);
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i)
      for (int q = 0; q < 3; ++q)
        for (int pp = 0; pp < 3; ++pp) {
          // node (i, j) at 3 j + i, mode (pp, q) at 3 q + pp
          co[(3 * j + i) * 9 + 3 * q + pp] = V[i][pp] * V[j][q];          // V2
          co[81 + (3 * q + pp) * 9 + 3 * j + i] = Vi[pp][i] * Vi[q][j];   // V2^{-1}
        }
  for (int q = 0; q < 3; ++q)
    for (int pp = 0; pp < 3; ++pp) co[162 + 3 * q + pp] = C.c * (lam[pp] + lam[q]);
  std::vector<float> cof(co.begin(), co.end());
  C.co = (double*)p; cudaMemcpy(p, co.data(), 171 * 8, cudaMemcpyHostToDevice); p += up(171 * 8);
  C.cof = (float*)p; cudaMemcpy(p, cof.data(), 171 * 4, cudaMemcpyHostToDevice); p += up(171 * 4);
  return p;
}

static void mg_slot_tables(const Geom& g, MgHost& h, unsigned char*& p);
static int tail_level(const MgHost& h);

cudaError_t mg_setup(Geom& g, void* ws, const double* a_edges, double a0) {
  // this translation unit's copy of the register-FFT twiddle table
  cudaError_t e0 = upload_w96();
  if (e0 != cudaSuccess) return e0;
  MgHost h;
  const bool neu = g.bc == PCB_BC_NEUMANN;
  h.nlev = levels_for(g.N, neu);
  if (h.nlev > kMaxLevels) return cudaErrorInvalidValue;
  h.nsys = g.n;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  unsigned char* p = (unsigned char*)ws;
  if (neu) {
    p = mg_setup_neumann(g, h, p, a0);
    mg_slot_tables(g, h, p);
    h.tail_l0 = tail_level(h);
    if ((size_t)(p - (unsigned char*)ws) > mg_workspace_bytes(g)) return cudaErrorInvalidValue;
    for (auto& e : registry())
      if (e.first == ws) { e.second = h; g.mg = ws; return cudaGetLastError(); }
    registry().push_back({ws, h});
    g.mg = ws;
    return cudaGetLastError();
  }
  // fine coefficients = tau/h^2 * a at the edges; coarser levels average the two fine edges each
  // coarse edge spans and are rescaled with their own spacing
  int N = g.N;
  std::vector<double> ax(a_edges, a_edges + (size_t)N * (N + 1));
  std::vector<double> ay(a_edges + (size_t)N * (N + 1), a_edges + 2 * (size_t)N * (N + 1));
  std::vector<unsigned char> hostbuf;
  for (int l = 0; l < h.nlev; ++l) {
    MgLevel& L = h.lev[l];
    std::memset(&L, 0, sizeof(L));
    L.N = N;
    const double hl = 1.0 / (N + 1), s = g.tau / (hl * hl);
    const size_t ne = (size_t)N * (N + 1), nn = (size_t)N * N;
    std::vector<double> axs(ne), ays(ne), dgs(nn);
    for (size_t k = 0; k < ne; ++k) { axs[k] = s * ax[k]; ays[k] = s * ay[k]; }
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i)
        dgs[(size_t)j * N + i] = axs[(size_t)j * (N + 1) + i] + axs[(size_t)j * (N + 1) + i + 1] +
                                 ays[(size_t)j * N + i] + ays[(size_t)(j + 1) * N + i];
    std::vector<float> axf(ne), ayf(ne), dgf(nn);
    for (size_t k = 0; k < ne; ++k) { axf[k] = (float)axs[k]; ayf[k] = (float)ays[k]; }
    for (size_t k = 0; k < nn; ++k) dgf[k] = (float)dgs[k];
    L.axs = (double*)p; cudaMemcpy(p, axs.data(), ne * 8, cudaMemcpyHostToDevice); p += up(ne * 8);
    L.ays = (double*)p; cudaMemcpy(p, ays.data(), ne * 8, cudaMemcpyHostToDevice); p += up(ne * 8);
    L.dgs = (double*)p; cudaMemcpy(p, dgs.data(), nn * 8, cudaMemcpyHostToDevice); p += up(nn * 8);
    L.axf = (float*)p; cudaMemcpy(p, axf.data(), ne * 4, cudaMemcpyHostToDevice); p += up(ne * 4);
    L.ayf = (float*)p; cudaMemcpy(p, ayf.data(), ne * 4, cudaMemcpyHostToDevice); p += up(ne * 4);
    L.dgf = (float*)p; cudaMemcpy(p, dgf.data(), nn * 4, cudaMemcpyHostToDevice); p += up(nn * 4);
    for (int k = 0; k < 3; ++k) { L.a[k] = p; p += up((size_t)h.nsys * nn * sizeof(double2)); }
    if (l == 0) {
      h.zfine = p; p += up((size_t)h.nsys * nn * sizeof(double2));
      h.xfine = p; p += up((size_t)h.nsys * nn * sizeof(double2));
    }
    if (N == 1) break;
    // coarse coefficients: coarse row J sits on fine row 2J+1 (0-based), coarse edge e spans fine
    // edges 2e and 2e+1 (and symmetrically for the x2 edges)
    const int Nc = (N - 1) / 2;
    std::vector<double> axc((size_t)Nc * (Nc + 1)), ayc((size_t)Nc * (Nc + 1));
    for (int J = 0; J < Nc; ++J)
      for (int e = 0; e <= Nc; ++e)
        axc[(size_t)J * (Nc + 1) + e] =
            0.5 * (ax[(size_t)(2 * J + 1) * (N + 1) + 2 * e] + ax[(size_t)(2 * J + 1) * (N + 1) + 2 * e + 1]);
    for (int e = 0; e <= Nc; ++e)
      for (int I = 0; I < Nc; ++I)
        ayc[(size_t)e * Nc + I] = 0.5 * (ay[(size_t)(2 * e) * N + 2 * I + 1] + ay[(size_t)(2 * e + 1) * N + 2 * I + 1]);
    ax.swap(axc); ay.swap(ayc);
    N = Nc;
  }
  mg_slot_tables(g, h, p);
  h.tail_l0 = tail_level(h);
  if ((size_t)(p - (unsigned char*)ws) > mg_workspace_bytes(g)) return cudaErrorInvalidValue;
  for (auto& e : registry())
    if (e.first == ws) { e.second = h; return cudaGetLastError(); }
  registry().push_back({ws, h});
  g.mg = ws;
  return cudaGetLastError();
}

// per-slot table from lambda(S_n) at the F-slots (same formula as the spectral tables)
static void mg_slot_tables(const Geom& g, MgHost& h, unsigned char*& p) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int n = g.n, half = n / 2;
  std::vector<double2> td((size_t)half * 4);
  std::vector<float2> tf((size_t)half * 4);
  for (int r = 0; r < half; ++r) {
    const double psi = -M_PI * (2.0 * r + 1.0) / n;
    const double c = std::cos(psi), s = std::sin(psi);
    const double f1r = 1.0 - c, f1i = -s;
    double f2r = g.theta + (1.0 - g.theta) * c, f2i = (1.0 - g.theta) * s;
    if (std::hypot(f2r, f2i) < 1e-14) { f2r = 1.0; f2i = 0.0; }
    const double den = f2r * f2r + f2i * f2i;
    const double mr = (f1r * f2r + f1i * f2i) / den, mi = (f1i * f2r - f1r * f2i) / den;
    const double a = g.alpha;
    const double sq = std::sqrt(mi * mi + a * a);
    // Lemma 3.14 (principal root): D1 = Re mu + i sqrt(Im^2 mu + alpha^2); M = -(i/alpha)(sq - Im mu)
    const double Mi = -(sq - mi) / a;                 // M = i * Mi (purely imaginary)
    const double inv = 1.0 / (1.0 + Mi * Mi);         // 1/(1 - M^2) with M^2 = -Mi^2
    td[4 * r + 0] = make_double2(mr, sq);             // D1
    td[4 * r + 1] = make_double2(0.0, Mi);            // M
    td[4 * r + 2] = make_double2(inv, 0.0);
    td[4 * r + 3] = make_double2(std::sqrt(mr * mr + mi * mi + a * a), 0.0);   // P_MS shift sigma_r
    for (int k = 0; k < 4; ++k) tf[4 * r + k] = make_float2((float)td[4 * r + k].x, (float)td[4 * r + k].y);
  }
  h.tab_d = (double2*)p; cudaMemcpy(p, td.data(), td.size() * sizeof(double2), cudaMemcpyHostToDevice);
  p += up(td.size() * sizeof(double2));
  h.tab_f = (float2*)p; cudaMemcpy(p, tf.data(), tf.size() * sizeof(float2), cudaMemcpyHostToDevice);
  p += up(tf.size() * sizeof(float2));
}

void mg_release(const void* ws) {
  auto& r = registry();
  for (size_t k = 0; k < r.size(); ++k)
    if (r[k].first == ws) { r.erase(r.begin() + k); return; }
}

// ------------------------------------------------------------------------------------------
// kernels (one instance; thread per (system, grid point)).  Blocks of 32 x 8 threads cover tiles
// of 32 x 8 points of one system's grid (grid x, y over the tiles, z over the systems), so that
// consecutive threads touch consecutive points and no index needs a division.
// ------------------------------------------------------------------------------------------
struct GridPt { int b, i, j; };
__device__ __forceinline__ GridPt grid_pt() {
  return GridPt{(int)blockIdx.z, (int)(blockIdx.x * 32 + threadIdx.x), (int)(blockIdx.y * 8 + threadIdx.y)};
}
static dim3 grid_for(int N, int nsys) { return dim3((unsigned)((N + 31) / 32), (unsigned)((N + 7) / 8), (unsigned)nsys); }
static const dim3 kMgBlock(32, 8);
template <typename R> struct Coef;
template <> struct Coef<float> {
  static __device__ const float* ax(const MgLevel& L) { return L.axf; }
  static __device__ const float* ay(const MgLevel& L) { return L.ayf; }
  static __device__ const float* dg(const MgLevel& L) { return L.dgf; }
};
template <> struct Coef<double> {
  static __device__ const double* ax(const MgLevel& L) { return L.axs; }
  static __device__ const double* ay(const MgLevel& L) { return L.ays; }
  static __device__ const double* dg(const MgLevel& L) { return L.dgs; }
};

// (tau K z) at point (i, j) of system b
template <typename R>
__device__ __forceinline__ cx<R> tauKz(const MgLevel& L, const cx<R>* __restrict__ z, int i, int j) {
  const int N = L.N;
  if (L.neu) {   // mirrored neighbours: u_{-1} = u_1, u_N = u_{N-2}
    const R c = sizeof(R) == 4 ? (R)L.cf : (R)L.c;
    const cx<R> l = z[j * N + (i > 0 ? i - 1 : 1)], r = z[j * N + (i < N - 1 ? i + 1 : N - 2)];
    const cx<R> d = z[(j > 0 ? j - 1 : 1) * N + i], t = z[(j < N - 1 ? j + 1 : N - 2) * N + i];
    const cx<R> nb = cadd(cadd(l, r), cadd(d, t));
    return cscale(csub(cscale(z[j * N + i], (R)4), nb), c);
  }
  const R* ax = Coef<R>::ax(L) + (long long)j * (N + 1);
  const R* ay = Coef<R>::ay(L);
  const cx<R> c = z[j * N + i];
  cx<R> s = mk<R>(0, 0);
  if (i > 0) s = cadd(s, cscale(z[j * N + i - 1], ax[i]));
  if (i < N - 1) s = cadd(s, cscale(z[j * N + i + 1], ax[i + 1]));
  if (j > 0) s = cadd(s, cscale(z[(j - 1) * N + i], ay[(long long)j * N + i]));
  if (j < N - 1) s = cadd(s, cscale(z[(j + 1) * N + i], ay[(long long)(j + 1) * N + i]));
  const R d = Coef<R>::dg(L)[j * N + i];
  return csub(cscale(c, d), s);
}

template <typename R>
__device__ __forceinline__ cx<R> shift_of(const cx<R>* __restrict__ tab, int b, int kind) {
  const int r = b >> 1;
  return kind == 2 ? tab[4 * r + 0] : mk<R>(tab[4 * r + 3].x, (R)0);
}

// Per-point operations, shared by the one-launch-per-step kernels of the fine levels and the
// fused kernel of the coarse levels (identical arithmetic on either path).  Arrays hold one
// system's grid, row j of N points at j N.

// Jacobi diagonal inverse of system shift mu at point pt
template <typename R>
__device__ __forceinline__ cx<R> jacobi_dinv(const MgLevel& L, cx<R> mu, int pt) {
  const R dgk = L.neu ? (R)4 * (sizeof(R) == 4 ? (R)L.cf : (R)L.c) : Coef<R>::dg(L)[pt];
  const cx<R> d = mk<R>(mu.x + dgk, mu.y);
  const R rd = (R)1 / (d.x * d.x + d.y * d.y);
  return mk<R>(d.x * rd, -d.y * rd);
}

// one damped Jacobi update at (i, j): out = z + w (rhs - A z) / diag (first: z = 0)
template <typename R>
__device__ __forceinline__ cx<R> jacobi_pt(const MgLevel& L, cx<R> mu, cx<R> dinv, const cx<R>* __restrict__ rhs,
                                           const cx<R>* __restrict__ z, int i, int j, bool first, R w) {
  const int pt = j * L.N + i;
  if (first) return cscale(cmul(rhs[pt], dinv), w);
  const cx<R> Az = cadd(cmul(mu, z[pt]), tauKz<R>(L, z, i, j));
  return cadd(z[pt], cscale(cmul(csub(rhs[pt], Az), dinv), w));
}

// residual rhs - A z at (i, j)
template <typename R>
__device__ __forceinline__ cx<R> resid_pt(const MgLevel& L, cx<R> mu, const cx<R>* __restrict__ rhs,
                                          const cx<R>* __restrict__ z, int i, int j) {
  const int pt = j * L.N + i;
  const cx<R> Az = cadd(cmul(mu, z[pt]), tauKz<R>(L, z, i, j));
  return csub(rhs[pt], Az);
}

// full weighting: coarse (I, J) <- fine 9-point neighbourhood of (2I+1, 2J+1) (0-based); Neumann:
// of (2I, 2J) with mirrored ghost values
template <typename R>
__device__ __forceinline__ cx<R> restrict_pt(int Nf, bool neu, const cx<R>* fb, int I, int J) {
  const int fi = neu ? 2 * I : 2 * I + 1, fj = neu ? 2 * J : 2 * J + 1;
  auto mir = [&](int k) { return k < 0 ? -k : (k > Nf - 1 ? 2 * (Nf - 1) - k : k); };
  auto at = [&](int ii, int jj) { return neu ? fb[mir(jj) * Nf + mir(ii)] : fb[jj * Nf + ii]; };
  cx<R> s = cscale(at(fi, fj), (R)4);
  s = cadd(s, cscale(cadd(cadd(at(fi - 1, fj), at(fi + 1, fj)), cadd(at(fi, fj - 1), at(fi, fj + 1))), (R)2));
  s = cadd(s, cadd(cadd(at(fi - 1, fj - 1), at(fi + 1, fj - 1)), cadd(at(fi - 1, fj + 1), at(fi + 1, fj + 1))));
  return cscale(s, (R)(1.0 / 16.0));
}

// bilinear prolongation of the coarse grid cb (Nc points per side) at fine (i, j).  Dirichlet:
// fine 0-based index 2K+1 sits on coarse node K, an even fine index between nodes K-1 and K; with
// Ka = (k-1) >> 1 and Kb = k >> 1 in each direction (equal for an odd k) the value is 1/4 of the
// sum over the four (Ka|Kb) pairs, which equals the one-, two- or four-node average exactly
// (scalings by powers of two), so no thread branches on the parity of its point.  Neumann: even
// fine nodes are coarse nodes.
template <typename R>
__device__ __forceinline__ cx<R> prolong_pt(int Nc, bool neu, const cx<R>* cb, int i, int j) {
  if (neu) {
    const int I0 = i >> 1, J0 = j >> 1, I1 = (i + 1) >> 1, J1 = (j + 1) >> 1;   // equal when even
    return cscale(cadd(cadd(cb[J0 * Nc + I0], cb[J0 * Nc + I1]), cadd(cb[J1 * Nc + I0], cb[J1 * Nc + I1])), (R)0.25);
  }
  const int Ia = (i - 1) >> 1, Ib = i >> 1, Ja = (j - 1) >> 1, Jb = j >> 1;
  const bool xa = Ia >= 0, xb = Ib < Nc, ya = Ja >= 0, yb = Jb < Nc;
  const cx<R> zero = mk<R>(0, 0);
  const cx<R> c11 = xa && ya ? cb[Ja * Nc + Ia] : zero, c21 = xb && ya ? cb[Ja * Nc + Ib] : zero;
  const cx<R> c12 = xa && yb ? cb[Jb * Nc + Ia] : zero, c22 = xb && yb ? cb[Jb * Nc + Ib] : zero;
  return cscale(cadd(cadd(c11, c21), cadd(c12, c22)), (R)0.25);
}

// Neumann 3 x 3 grid: exact solve z = V2 diag(1/(mu + lambda)) V2^{-1} rhs at `node`
template <typename R>
__device__ __forceinline__ cx<R> coarse_neu_pt(const MgLevel& L, cx<R> mu, const cx<R>* rb, int node) {
  const R* co = sizeof(R) == 4 ? (const R*)L.cof : (const R*)L.co;
  cx<R> acc = mk<R>(0, 0);
  for (int md = 0; md < 9; ++md) {
    cx<R> w = mk<R>(0, 0);
    for (int k = 0; k < 9; ++k) w = cadd(w, cscale(rb[k], co[81 + md * 9 + k]));
    const cx<R> den = mk<R>(mu.x + co[162 + md], mu.y);
    const R dd = den.x * den.x + den.y * den.y;
    w = cmul(w, mk<R>(den.x / dd, -den.y / dd));
    acc = cadd(acc, cscale(w, co[node * 9 + md]));
  }
  return acc;
}

// The two systems of a frequency slot (2r and 2r + 1) share the shift and hence the diagonal:
// a thread treats one grid point of both (grid z runs over the slots).

template <typename R, bool FIRST>
__global__ void __launch_bounds__(256) k_mg_jacobi(MgLevel L, const cx<R>* __restrict__ tab, int kind,
                                                   const cx<R>* __restrict__ rhs, const cx<R>* __restrict__ z,
                                                   cx<R>* __restrict__ out, R w) {
  const int N = L.N, nn = N * N;
  const GridPt q = grid_pt();
  if (q.i >= N || q.j >= N) return;
  const int b = 2 * q.b, pt = q.j * N + q.i;
  const cx<R> mu = shift_of<R>(tab, b, kind);
  const cx<R> dinv = jacobi_dinv<R>(L, mu, pt);
  const long long o0 = (long long)b * nn, o1 = o0 + nn;
  if (FIRST) {
    const cx<R> r0 = rhs[o0 + pt], r1 = rhs[o1 + pt];
    out[o0 + pt] = cscale(cmul(r0, dinv), w);
    out[o1 + pt] = cscale(cmul(r1, dinv), w);
    return;
  }
  // jacobi_pt's arithmetic, with both systems' products formed before either update so that all
  // loads are in flight together
  const cx<R> Az0 = cadd(cmul(mu, z[o0 + pt]), tauKz<R>(L, z + o0, q.i, q.j));
  const cx<R> Az1 = cadd(cmul(mu, z[o1 + pt]), tauKz<R>(L, z + o1, q.i, q.j));
  const cx<R> n0 = cadd(z[o0 + pt], cscale(cmul(csub(rhs[o0 + pt], Az0), dinv), w));
  const cx<R> n1 = cadd(z[o1 + pt], cscale(cmul(csub(rhs[o1 + pt], Az1), dinv), w));
  out[o0 + pt] = n0;
  out[o1 + pt] = n1;
}

template <typename R>
__global__ void __launch_bounds__(256) k_mg_resid(MgLevel L, const cx<R>* __restrict__ tab, int kind,
                                                  const cx<R>* __restrict__ rhs, const cx<R>* __restrict__ z,
                                                  cx<R>* __restrict__ res) {
  const int N = L.N, nn = N * N;
  const GridPt q = grid_pt();
  if (q.i >= N || q.j >= N) return;
  const int b = 2 * q.b, pt = q.j * N + q.i;
  const cx<R> mu = shift_of<R>(tab, b, kind);
  const long long o0 = (long long)b * nn, o1 = o0 + nn;
  const cx<R> r0 = resid_pt<R>(L, mu, rhs + o0, z + o0, q.i, q.j);
  const cx<R> r1 = resid_pt<R>(L, mu, rhs + o1, z + o1, q.i, q.j);
  res[o0 + pt] = r0;
  res[o1 + pt] = r1;
}

// tau K z at grid point (gi, gj) of a Dirichlet level from a shared-memory window whose row
// pitch is WX and in which (gi, gj) sits at (li, lj): the arithmetic of tauKz
template <typename R>
__device__ __forceinline__ cx<R> tauKz_win(const MgLevel& L, const cx<R>* zs, int WX, int li, int lj, int gi,
                                           int gj) {
  const int N = L.N;
  const R* ax = Coef<R>::ax(L) + (long long)gj * (N + 1);
  const R* ay = Coef<R>::ay(L);
  const cx<R> c = zs[lj * WX + li];
  cx<R> s = mk<R>(0, 0);
  if (gi > 0) s = cadd(s, cscale(zs[lj * WX + li - 1], ax[gi]));
  if (gi < N - 1) s = cadd(s, cscale(zs[lj * WX + li + 1], ax[gi + 1]));
  if (gj > 0) s = cadd(s, cscale(zs[(lj - 1) * WX + li], ay[(long long)gj * N + gi]));
  if (gj < N - 1) s = cadd(s, cscale(zs[(lj + 1) * WX + li], ay[(long long)(gj + 1) * N + gi]));
  const R d = Coef<R>::dg(L)[gj * N + gi];
  return csub(cscale(c, d), s);
}

// The pre-smoothing of a Dirichlet level (two sweeps, the first from zero) and the residual of its
// result in one launch.  A block takes a 32 x 8 tile of both systems of a slot: it loads the
// right-hand sides on the tile with a halo of two points, runs the first sweep there, the second on
// the tile with a halo of one, and forms the residual on the tile, all in shared memory; it writes
// the smoothed solution and the residual.  The same per-point arithmetic as the three separate
// launches (jacobi_pt, resid_pt), which read and wrote 8 full grids where this moves 3.
template <typename R>
__global__ void __launch_bounds__(256) k_mg_presmooth(MgLevel L, const cx<R>* __restrict__ tab, int kind,
                                                      const cx<R>* __restrict__ rhs, cx<R>* __restrict__ zout,
                                                      cx<R>* __restrict__ res, R w) {
  using C = cx<R>;
  constexpr int TX = 32, TY = 8, WX2 = TX + 4, WY2 = TY + 4, WX1 = TX + 2, WY1 = TY + 2;
  __shared__ C r2[2][WX2 * WY2], z1[2][WX2 * WY2], z2[2][WX1 * WY1];
  const int N = L.N, nn = N * N;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, tid = threadIdx.y * TX + threadIdx.x;
  const int b = 2 * blockIdx.z;
  const C mu = shift_of<R>(tab, b, kind);
  const long long o0 = (long long)b * nn;
  const C zero = mk<R>(0, 0);
  // the right-hand sides and the first sweep (from zero) on the tile with a halo of 2
  for (int e = tid; e < WX2 * WY2; e += TX * TY) {
    const int lj = e / WX2, li = e - lj * WX2, gi = x0 - 2 + li, gj = y0 - 2 + lj;
    const bool in = gi >= 0 && gi < N && gj >= 0 && gj < N;
    const C dinv = in ? jacobi_dinv<R>(L, mu, gj * N + gi) : zero;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const C rv = in ? rhs[o0 + (long long)k * nn + gj * N + gi] : zero;
      r2[k][e] = rv;
      z1[k][e] = in ? cscale(cmul(rv, dinv), w) : zero;
    }
  }
  __syncthreads();
  // the second sweep on the tile with a halo of 1
  for (int e = tid; e < WX1 * WY1; e += TX * TY) {
    const int lj1 = e / WX1, li1 = e - lj1 * WX1, gi = x0 - 1 + li1, gj = y0 - 1 + lj1;
    const int li = li1 + 1, lj = lj1 + 1;
    const bool in = gi >= 0 && gi < N && gj >= 0 && gj < N;
    const C dinv = in ? jacobi_dinv<R>(L, mu, gj * N + gi) : zero;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      C v = zero;
      if (in) {
        const C zc = z1[k][lj * WX2 + li];
        const C Az = cadd(cmul(mu, zc), tauKz_win<R>(L, z1[k], WX2, li, lj, gi, gj));
        v = cadd(zc, cscale(cmul(csub(r2[k][lj * WX2 + li], Az), dinv), w));
      }
      z2[k][e] = v;
    }
  }
  __syncthreads();
  // the tile: the smoothed solution and its residual
  const int gi = x0 + threadIdx.x, gj = y0 + threadIdx.y;
  if (gi < N && gj < N) {
    const int li1 = threadIdx.x + 1, lj1 = threadIdx.y + 1, pt = gj * N + gi;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const C zc = z2[k][lj1 * WX1 + li1];
      const C Az = cadd(cmul(mu, zc), tauKz_win<R>(L, z2[k], WX1, li1, lj1, gi, gj));
      zout[o0 + (long long)k * nn + pt] = zc;
      res[o0 + (long long)k * nn + pt] = csub(r2[k][(threadIdx.y + 2) * WX2 + threadIdx.x + 2], Az);
    }
  }
}

template <typename R, bool NEU>
__global__ void __launch_bounds__(256) k_mg_restrict(int Nf, const cx<R>* __restrict__ f, cx<R>* __restrict__ c) {
  const int Nc = NEU ? (Nf + 1) / 2 : (Nf - 1) / 2, nnc = Nc * Nc, nnf = Nf * Nf;
  const GridPt q = grid_pt();
  if (q.i >= Nc || q.j >= Nc) return;
  const cx<R> v0 = restrict_pt<R>(Nf, NEU, f + 2LL * q.b * nnf, q.i, q.j);
  const cx<R> v1 = restrict_pt<R>(Nf, NEU, f + (2LL * q.b + 1) * nnf, q.i, q.j);
  c[2LL * q.b * nnc + q.j * Nc + q.i] = v0;
  c[(2LL * q.b + 1) * nnc + q.j * Nc + q.i] = v1;
}

// the prolonged coarse correction added to the fine solution
template <typename R, bool NEU>
__global__ void __launch_bounds__(256) k_mg_prolong_add(int Nf, const cx<R>* __restrict__ c, cx<R>* __restrict__ z) {
  const int Nc = NEU ? (Nf + 1) / 2 : (Nf - 1) / 2, nnc = Nc * Nc, nnf = Nf * Nf;
  const GridPt q = grid_pt();
  if (q.i >= Nf || q.j >= Nf) return;
  const long long o0 = 2LL * q.b * nnf + q.j * Nf + q.i, o1 = o0 + nnf;
  const cx<R> v0 = prolong_pt<R>(Nc, NEU, c + 2LL * q.b * nnc, q.i, q.j);
  const cx<R> v1 = prolong_pt<R>(Nc, NEU, c + (2LL * q.b + 1) * nnc, q.i, q.j);
  const cx<R> z0 = z[o0], z1 = z[o1];
  z[o0] = cadd(z0, v0);
  z[o1] = cadd(z1, v1);
}

// Neumann 3 x 3 grid, one thread per (system, node)
template <typename R>
__global__ void k_mg_coarse_neu(MgLevel L, int nsys, const cx<R>* __restrict__ tab, int kind,
                                const cx<R>* __restrict__ rhs, cx<R>* __restrict__ z) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)nsys * 9) return;
  const int b = (int)(idx / 9), node = (int)(idx - (long long)b * 9);
  z[(long long)b * 9 + node] = coarse_neu_pt<R>(L, shift_of<R>(tab, b, kind), rhs + (long long)b * 9, node);
}

// ------------------------------------------------------------------------------------------
// The coarse levels in one launch.  Below about 33 points per side a level's steps are too small
// to fill the GPU, and each one-per-step launch costs several microseconds whatever its size.
// One block takes both systems of a slot through the V-cycle from level l0 down to the coarsest
// grid and back, with every level's right-hand side, solution and spare grid in shared memory,
// the same per-point arithmetic as the fine levels, and a block barrier between steps.
// ------------------------------------------------------------------------------------------
struct MgTail {
  MgLevel lev[kMaxLevels];
  int l0, nlev;
};

template <typename R>
size_t tail_smem(const MgTail& t) {
  size_t e = 0;
  for (int l = t.l0; l < t.nlev; ++l) e += 3 * 2 * (size_t)t.lev[l].N * t.lev[l].N;
  return e * sizeof(cx<R>);
}

static constexpr size_t kTailSmemMax = 200 * 1024;
static_assert(kNu % 2 == 0, "the fused coarse levels expect the pre-smoothing to end in z");

// first level of the fused launch: the first below the finest with at most 33 points per side whose
// levels fit the shared-memory budget in FP64; -1 if none
static int tail_level(const MgHost& h) {
  for (int l = 1; l < h.nlev; ++l) {
    if (h.lev[l].N > 33) continue;
    MgTail T;
    for (int k = 0; k < h.nlev; ++k) T.lev[k] = h.lev[k];
    T.l0 = l; T.nlev = h.nlev;
    return tail_smem<double>(T) <= kTailSmemMax ? l : -1;
  }
  return -1;
}

template <typename R>
__global__ void __launch_bounds__(256) k_mg_vcycle_tail(MgTail T, const cx<R>* __restrict__ tab, int kind,
                                                        const cx<R>* __restrict__ grhs, cx<R>* __restrict__ gz) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* base[kMaxLevels][3];                         // [level][rhs, z, spare], each 2 systems x N^2
  {
    C* p = (C*)smem_raw;
    for (int l = T.l0; l < T.nlev; ++l) {
      const int nn2 = 2 * T.lev[l].N * T.lev[l].N;
      for (int a = 0; a < 3; ++a) { base[l][a] = p; p += nn2; }
    }
  }
  const int slot = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const cx<R> mu = shift_of<R>(tab, 2 * slot, kind);
  const R w = (R)kJacobiWeight;
  {   // right-hand sides of level l0
    const int nn = T.lev[T.l0].N * T.lev[T.l0].N;
    const C* src = grhs + (long long)2 * slot * nn;
    for (int e = tid; e < 2 * nn; e += nt) base[T.l0][0][e] = src[e];
  }
  __syncthreads();
  // sweep over every (system, point) of level l
  auto each = [&](int l, auto&& f) {
    const int N = T.lev[l].N, nn = N * N;
    for (int e = tid; e < 2 * nn; e += nt) {
      const int k = e >= nn ? 1 : 0, pt = e - k * nn, j = pt / N, i = pt - j * N;
      f(k, pt, i, j, nn);
    }
    __syncthreads();
  };
  // descent: nu1 sweeps (the first from zero, into `spare`, so that the last post-smoothing
  // sweep lands in z), residual, restriction
  for (int l = T.l0; l < T.nlev - 1; ++l) {
    const MgLevel& L = T.lev[l];
    C* rhs = base[l][0];
    C* cur = base[l][2];
    C* oth = base[l][1];
    each(l, [&](int k, int pt, int i, int j, int nn) {
      cur[k * nn + pt] = jacobi_pt<R>(L, mu, jacobi_dinv<R>(L, mu, pt), rhs + k * nn, nullptr, i, j, true, w);
    });
    for (int s = 1; s < kNu; ++s) {
      each(l, [&](int k, int pt, int i, int j, int nn) {
        oth[k * nn + pt] = jacobi_pt<R>(L, mu, jacobi_dinv<R>(L, mu, pt), rhs + k * nn, cur + k * nn, i, j, false, w);
      });
      C* t = cur; cur = oth; oth = t;
    }
    each(l, [&](int k, int pt, int i, int j, int nn) {
      oth[k * nn + pt] = resid_pt<R>(L, mu, rhs + k * nn, cur + k * nn, i, j);
    });
    each(l + 1, [&](int k, int pt, int i, int j, int nn) {
      base[l + 1][0][k * nn + pt] = restrict_pt<R>(L.N, L.neu != 0, oth + k * L.N * L.N, i, j);
    });
  }
  {   // coarsest grid: exact solve
    const int l = T.nlev - 1;
    const MgLevel& L = T.lev[l];
    C* rhs = base[l][0];
    C* z = base[l][1];
    each(l, [&](int k, int pt, int i, int j, int nn) {
      z[k * nn + pt] = L.neu ? coarse_neu_pt<R>(L, mu, rhs + k * nn, pt)
                             : jacobi_pt<R>(L, mu, jacobi_dinv<R>(L, mu, pt), rhs + k * nn, nullptr, i, j, true, (R)1);
    });
  }
  // ascent: prolongation added into z, nu2 sweeps ending in z
  for (int l = T.nlev - 2; l >= T.l0; --l) {
    const MgLevel& L = T.lev[l];
    const int Nc = T.lev[l + 1].N;
    C* rhs = base[l][0];
    C* cur = base[l][1];
    C* oth = base[l][2];
    each(l, [&](int k, int pt, int i, int j, int nn) {
      cur[k * nn + pt] = cadd(cur[k * nn + pt], prolong_pt<R>(Nc, L.neu != 0, base[l + 1][1] + k * Nc * Nc, i, j));
    });
    for (int s = 0; s < kNu; ++s) {
      each(l, [&](int k, int pt, int i, int j, int nn) {
        oth[k * nn + pt] = jacobi_pt<R>(L, mu, jacobi_dinv<R>(L, mu, pt), rhs + k * nn, cur + k * nn, i, j, false, w);
      });
      C* t = cur; cur = oth; oth = t;
    }
  }
  {   // solution of level l0
    const int nn = T.lev[T.l0].N * T.lev[T.l0].N;
    C* dst = gz + (long long)2 * slot * nn;
    for (int e = tid; e < 2 * nn; e += nt) dst[e] = base[T.l0][1][e];
  }
}

// a += b  or  a = b (copy)
template <typename R>
__global__ void k_mg_axpy(long long len, const cx<R>* __restrict__ src, cx<R>* __restrict__ dst, int copy) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= len) return;
  dst[idx] = copy ? src[idx] : cadd(dst[idx], src[idx]);
}

// ------------------------------------------------------------------------------------------
// time passes around the multigrid
// ------------------------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ const cx<R>* twt_(const Geom& g);
template <> __device__ __forceinline__ const float2* twt_<float>(const Geom& g) { return g.twt_f; }
template <> __device__ __forceinline__ const double2* twt_<double>(const Geom& g) { return g.twt_d; }
template <typename R> __device__ __forceinline__ const cx<R>* pre_(const Geom& g);
template <> __device__ __forceinline__ const float2* pre_<float>(const Geom& g) { return g.pre_f; }
template <> __device__ __forceinline__ const double2* pre_<double>(const Geom& g) { return g.pre_d; }

__host__ __device__ __forceinline__ int padded_len_mg(int len) { return (len + (len >> 5) + 1) | 1; }

// Shared-memory radix-2 Stockham-free DFT of one column of length n by a single warp-group:
// the time passes here handle one column per warp with the register/shuffle FFT.
template <typename R, int Q>
__device__ __forceinline__ void col_fft(cx<R>* line, int t, int P, const cx<R>* __restrict__ tw, bool inv) {
  using T = cx<R>;
  LaneStages<T, R> st;
  lane_stages<T, R>(st, t, P, inv);
  T x[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) x[q] = line[pidx(t + P * q)];
  __syncwarp();
  reg_dft<T, R, Q>(x, inv);
#pragma unroll
  for (int k1 = 1; k1 < Q; ++k1) {
    T w = __ldg(&tw[t * k1]);
    if (inv) w.y = -w.y;
    x[pos<Q>(k1)] = cmul(x[pos<Q>(k1)], w);
  }
  lane_dif<T, R, Q>(x, P, st);
  __syncwarp();
  const int k2 = bitrev(t, P);
#pragma unroll
  for (int k1 = 0; k1 < Q; ++k1) line[pidx(k1 + Q * k2)] = x[pos<Q>(k1)];
  __syncwarp();
}

// forward: v (FP64, 2 halves) -> right-hand sides of the n systems (slot r < n/2: 2r and 2r+1)
template <typename R, int Q>
__global__ void __launch_bounds__(256) k_mg_time_fwd(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                     int in_slot, const cx<R>* __restrict__ tab, int kind,
                                                     cx<R>* __restrict__ rhs, int cpw) {
  using T = cx<R>;
  const Geom& g = G[0];
  const int n = g.n, m = g.m, ls = padded_len_mg(n);
  const long long mn = g.mn;
  const double* __restrict__ x = S[0].v[in_slot];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = (T*)smem_raw;
  const int P = n / Q, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lpw = 32 / P;
  const int t = lane % P;
  const int cols_per_block = (blockDim.x >> 5) * lpw * cpw;
  const int c0 = blockIdx.x * cols_per_block;
  for (int e = threadIdx.x; e < cols_per_block * n; e += blockDim.x) {
    const int tt = e / cols_per_block, l = e - tt * cols_per_block;
    const int col = c0 + l;
    T v = mk<R>(0, 0);
    if (col < m) {
      const long long a = (long long)tt * m + col;
      v = cmul(mk<R>((R)x[a], (R)x[mn + a]), __ldg(&pre_<R>(g)[tt]));
    }
    tile[l * ls + pidx(tt)] = v;
  }
  __syncthreads();
  const int half = n / 2;
  for (int k = 0; k < cpw; ++k) {
    const int l = (warp * cpw + k) * lpw + lane / P;
    T* line = tile + l * ls;
    col_fft<R, Q>(line, t, P, twt_<R>(g), false);
    const int col = c0 + l;
    if (col < m) {
      for (int r = t; r < half; r += P) {
        const T Cr = line[pidx(r)], Cq = cconj(line[pidx(n - 1 - r)]);
        const T F1 = cscale(cadd(Cr, Cq), (R)0.5);
        const T F2 = cmul_mi(cscale(csub(Cr, Cq), (R)0.5));
        T T1 = F1, T2 = F2;
        if (kind == 2) {   // W^{-1} [F1; F2], W = [[1, M], [M, 1]]
          const T M = tab[4 * r + 1];
          const R inv = tab[4 * r + 2].x;
          T1 = cscale(csub(F1, cmul(M, F2)), inv);
          T2 = cscale(csub(F2, cmul(M, F1)), inv);
          T2 = cconj(T2);   // second component: solved as the conjugate system with D1
        }
        rhs[(long long)(2 * r) * m + col] = T1;
        rhs[(long long)(2 * r + 1) * m + col] = T2;
      }
    }
  }
}

// inverse: solutions of the n systems -> P^{-1} v (FP64, 2 halves)
template <typename R, int Q>
__global__ void __launch_bounds__(256) k_mg_time_inv(const Geom* __restrict__ G, const Slots* __restrict__ S,
                                                     int out_slot, const cx<R>* __restrict__ tab, int kind,
                                                     const cx<R>* __restrict__ z, int cpw) {
  using T = cx<R>;
  const Geom& g = G[0];
  const int n = g.n, m = g.m, ls = padded_len_mg(n);
  const long long mn = g.mn;
  double* __restrict__ y = S[0].v[out_slot];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = (T*)smem_raw;
  const int P = n / Q, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lpw = 32 / P;
  const int t = lane % P;
  const int cols_per_block = (blockDim.x >> 5) * lpw * cpw;
  const int c0 = blockIdx.x * cols_per_block;
  const int half = n / 2;
  for (int e = threadIdx.x; e < cols_per_block * half; e += blockDim.x) {
    const int r = e / cols_per_block, l = e - r * cols_per_block;
    const int col = c0 + l;
    T U1 = mk<R>(0, 0), U2 = mk<R>(0, 0);
    if (col < m) {
      const T Z1 = z[(long long)(2 * r) * m + col];
      T Z2 = z[(long long)(2 * r + 1) * m + col];
      if (kind == 2) {
        Z2 = cconj(Z2);
        const T M = tab[4 * r + 1];
        U1 = cadd(Z1, cmul(M, Z2));
        U2 = cadd(cmul(M, Z1), Z2);
      } else {
        U1 = Z1; U2 = Z2;
      }
    }
    tile[l * ls + pidx(r)] = cadd(U1, cmul_pi(U2));
    tile[l * ls + pidx(n - 1 - r)] = cadd(cconj(U1), cmul_pi(cconj(U2)));
  }
  __syncthreads();
  for (int k = 0; k < cpw; ++k) {
    const int l = (warp * cpw + k) * lpw + lane / P;
    col_fft<R, Q>(tile + l * ls, t, P, twt_<R>(g), true);
  }
  __syncthreads();
  const R sc = (R)1 / (R)n;
  for (int e = threadIdx.x; e < cols_per_block * n; e += blockDim.x) {
    const int tt = e / cols_per_block, l = e - tt * cols_per_block;
    const int col = c0 + l;
    if (col < m) {
      const T v = cscale(cmul(tile[l * ls + pidx(tt)], cconj(__ldg(&pre_<R>(g)[tt]))), sc);
      const long long a = (long long)tt * m + col;
      y[a] = (double)v.x;
      y[mn + a] = (double)v.y;
    }
  }
}

// ------------------------------------------------------------------------------------------
// host orchestration
// ------------------------------------------------------------------------------------------
static unsigned blocks_for(long long len) { return (unsigned)((len + 255) / 256); }

template <typename R>
static void vcycle(const MgHost& h, const cx<R>* tab, int kind, int l, const cx<R>* rhs, cx<R>* z, cx<R>* spare,
                   cudaStream_t st) {
  const MgLevel& L = h.lev[l];
  if (l > 0 && l == h.tail_l0) {      // the coarse levels in one launch, one block per slot
    MgTail T;
    for (int k = 0; k < h.nlev; ++k) T.lev[k] = h.lev[k];
    T.l0 = l; T.nlev = h.nlev;
    static DeviceOnce once;
    set_smem_limit(once, k_mg_vcycle_tail<R>, (int)kTailSmemMax);
    k_mg_vcycle_tail<R><<<h.nsys / 2, 256, tail_smem<R>(T), st>>>(T, tab, kind, rhs, z);
    g_mg_launches += 1;
    return;
  }
  const dim3 grids = grid_for(L.N, h.nsys / 2);     // one slot (two systems) per grid z
  const R w = (R)kJacobiWeight;
  if (l == h.nlev - 1) {
    if (L.neu) k_mg_coarse_neu<R><<<blocks_for((long long)h.nsys * 9), 256, 0, st>>>(L, h.nsys, tab, kind, rhs, z);
    else        // exact solve on the single-unknown grid: z = rhs / diag
      k_mg_jacobi<R, true><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, nullptr, z, (R)1);
    g_mg_launches += 1;
    return;
  }
  // pre-smoothing from zero: the first sweep z1 = w D^{-1} rhs, then nu1 - 1 sweeps ping-ponging
  // between `spare` and z.  The nu1 + nu2 = 2 nu sweeps alternate between the two buffers, so
  // starting in `spare` leaves the last post-smoothing sweep in z.
  cx<R>* cur = spare;
  cx<R>* oth = z;
  if (!L.neu && kNu == 2 && sizeof(R) == 4) {
    // both sweeps and the residual in one launch: the solution in z, the residual in `spare`.
    // FP32 only: the fused kernel repeats the sweeps on its halos, and in FP64, whose kernels are
    // bound by the FP64 rate rather than by memory, that costs more than it saves (level 0 at
    // N = 255, n = 256: 2.32 ms fused against about 1.9 ms for the three launches)
    k_mg_presmooth<R><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, z, spare, w);
    cur = z; oth = spare;
    g_mg_launches += 1;
  } else {
    k_mg_jacobi<R, true><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, nullptr, cur, w);
    for (int s = 1; s < kNu; ++s) {
      k_mg_jacobi<R, false><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, cur, oth, w);
      std::swap(cur, oth);
    }
    k_mg_resid<R><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, cur, oth);
    g_mg_launches += kNu + 1;
  }
  // restrict the residual to the coarse right-hand side
  const MgLevel& C = h.lev[l + 1];
  const dim3 gridc = grid_for(C.N, h.nsys / 2);
  cx<R>* crhs = (cx<R>*)C.a[0];
  if (L.neu) k_mg_restrict<R, true><<<gridc, kMgBlock, 0, st>>>(L.N, oth, crhs);
  else k_mg_restrict<R, false><<<gridc, kMgBlock, 0, st>>>(L.N, oth, crhs);
  vcycle<R>(h, tab, kind, l + 1, crhs, (cx<R>*)C.a[1], (cx<R>*)C.a[2], st);
  if (L.neu) k_mg_prolong_add<R, true><<<grids, kMgBlock, 0, st>>>(L.N, (const cx<R>*)C.a[1], cur);
  else k_mg_prolong_add<R, false><<<grids, kMgBlock, 0, st>>>(L.N, (const cx<R>*)C.a[1], cur);
  for (int s = 0; s < kNu; ++s) {
    k_mg_jacobi<R, false><<<grids, kMgBlock, 0, st>>>(L, tab, kind, rhs, cur, oth, w);
    std::swap(cur, oth);
  }
  g_mg_launches += kNu + 2;
  if (cur != z) {
    const long long len = (long long)h.nsys * L.N * L.N;
    k_mg_axpy<R><<<blocks_for(len), 256, 0, st>>>(len, cur, z, 1);
    g_mg_launches += 1;
  }
}

template <typename R, int Q>
static cudaError_t mg_apply(const Batch& B, const Geom& g, const MgHost& h, int kind, int cycles, int in_slot,
                            int out_slot) {
  using T = cx<R>;
  cudaStream_t st = B.stream;
  const T* tab = (const T*)(sizeof(R) == 4 ? (const void*)h.tab_f : (const void*)h.tab_d);
  const MgLevel& F = h.lev[0];
  const long long len = (long long)h.nsys * F.N * F.N;
  T* r0 = (T*)F.a[0];
  T* z0 = (T*)h.zfine;
  T* x0 = (T*)h.xfine;
  const int P = g.n / Q, lpw = 32 / P, cpw = 2;   // two lines per warp: 16-column tiles, 128-byte runs of FP64
  const int cols = 8 * lpw * cpw;
  const size_t smem = (size_t)cols * padded_len_mg(g.n) * sizeof(T);
  static DeviceOnce once;
  once([] {
    cudaFuncSetAttribute(k_mg_time_fwd<R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return cudaFuncSetAttribute(k_mg_time_inv<R, Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  const unsigned tb = (unsigned)((g.m + cols - 1) / cols);
  k_mg_time_fwd<R, Q><<<tb, 256, smem, st>>>(B.G, B.S, in_slot, tab, kind, r0, cpw);
  g_mg_launches += 2;
  for (int c = 0; c < cycles; ++c) {
    if (c == 0) {
      vcycle<R>(h, tab, kind, 0, r0, z0, (T*)F.a[1], st);
    } else {
      k_mg_resid<R><<<grid_for(F.N, h.nsys / 2), kMgBlock, 0, st>>>(F, tab, kind, r0, z0, x0);
      vcycle<R>(h, tab, kind, 0, x0, (T*)F.a[2], (T*)F.a[1], st);
      k_mg_axpy<R><<<blocks_for(len), 256, 0, st>>>(len, (const T*)F.a[2], z0, 0);
      g_mg_launches += 2;
    }
  }
  k_mg_time_inv<R, Q><<<tb, 256, smem, st>>>(B.G, B.S, out_slot, tab, kind, z0, cpw);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t mg_dispatch(const Batch& B, const Geom& g, const MgHost& h, int kind, int cycles, int in_slot,
                               int out_slot) {
  switch (g.time_q) {
    case 1: return mg_apply<R, 1>(B, g, h, kind, cycles, in_slot, out_slot);
    case 2: return mg_apply<R, 2>(B, g, h, kind, cycles, in_slot, out_slot);
    case 4: return mg_apply<R, 4>(B, g, h, kind, cycles, in_slot, out_slot);
    case 8: return mg_apply<R, 8>(B, g, h, kind, cycles, in_slot, out_slot);
    case 16: return mg_apply<R, 16>(B, g, h, kind, cycles, in_slot, out_slot);
    default: return cudaErrorInvalidValue;
  }
}

int mg_launch_count(int kind) { (void)kind; return 0; }
long long mg_launch_total() { return g_mg_launches; }

cudaError_t launch_precond_mg(const Batch& B, const Geom& g, int kind, int prec, int cycles, int in_slot,
                              int out_slot) {
  if (B.count != 1 || !g.mg) return cudaErrorInvalidValue;
  const MgHost* h = find_host(g.mg);
  if (!h) return cudaErrorInvalidValue;
  if (kind != PCB_PREC_PS && kind != PCB_PREC_PMS) return cudaErrorInvalidValue;
  return prec == PCB_MIXED ? mg_dispatch<float>(B, g, *h, kind, cycles, in_slot, out_slot)
                           : mg_dispatch<double>(B, g, *h, kind, cycles, in_slot, out_slot);
}

}  // namespace pcb
