/*
 * pcb.h -- C ABI of the block omega-circulant preconditioned all-at-once solver for
 * theta-discretised parabolic optimal control (Fung & Hon, "Block omega-circulant
 * preconditioners for parabolic optimal control problems"), for one NVIDIA GB300 (sm_103a).
 *
 * Problem (Sec. 1 of the paper): 2D heat-equation tracking problem on the unit square,
 * zero Dirichlet data, 5-point finite differences (M = I, K = -L), theta-scheme in time.
 * N interior points per side (m = N*N, h = 1/(N+1)), n time steps (tau = T/n),
 * regularisation gamma, alpha = tau/sqrt(gamma), omega = exp(i zeta).
 *
 * Vector layout (all "x", "b", "y" vectors, FP64, device memory, length 2*m*n):
 *   index = half*m*n + t*m + (i-1) + (j-1)*N,   t = 0..n-1, i, j = 1..N (x1 fastest).
 * For the symmetric system A (Eq. main_system) half 0 holds sqrt(gamma)*y~, half 1 holds p~;
 * the right-hand side is [g; sqrt(gamma) f].  For the nonsymmetric system A_hat
 * (Eq. main_system_nonsym) the unknowns are the same and the right-hand side is
 * [sqrt(gamma) f; g].
 *
 * Conventions for every entry point:
 *   - Return value: PCB_OK (0) on success, a negative PCB_ERR_* code on failure, or the positive
 *     PCB_NOT_CONVERGED when a solve ran out of iterations (x then holds the last iterate).
 *     No exception or abort crosses this boundary; pcb_status_str() names each code.
 *   - Pointers named *_dev are device pointers owned by the caller; they must stay valid until the
 *     work queued on the problem's stream has finished.  Host pointers (*_host, a_edges) are read
 *     during the call only.
 *   - All work is queued on the stream given at creation (NULL = legacy default stream); calls
 *     return without synchronising except pcb_solve (which waits for convergence tests) and
 *     the *_host variants (which copy through host memory).
 *   - A problem handle is used by one host thread at a time.
 *   - The library owns its workspaces (allocated in pcb_create, freed in pcb_destroy).
 */
#ifndef PCB_H
#define PCB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define PCB_OK 0
#define PCB_NOT_CONVERGED 1          /* solve stopped at maxit; x holds the last iterate        */
#define PCB_ERR_INVALID_ARG (-1)     /* N < 1, n < 2, theta outside [1/2, 1], gamma <= 0, ...   */
#define PCB_ERR_UNSUPPORTED (-2)     /* valid input this build does not handle (see pcb_create) */
#define PCB_ERR_SINGULAR (-3)        /* singular S^(2) and the remedy was disabled              */
#define PCB_ERR_OUT_OF_MEMORY (-4)   /* a workspace allocation failed                          */
#define PCB_ERR_CUDA (-5)            /* a CUDA runtime call failed                              */
#define PCB_ERR_NONFINITE (-6)       /* NaN or Inf in a right-hand side or during a solve       */
#define PCB_ERR_BREAKDOWN (-7)       /* MINRES met a non-positive preconditioned norm           */
#define PCB_ERR_TIMEOUT (-8)         /* a bounded device-side wait gave up                      */
#define PCB_ERR_TOO_LARGE (-9)       /* request exceeds a documented size limit                 */

/* ---- enumerations ---------------------------------------------------------------------- */
enum pcb_precision { PCB_FP64 = 0, PCB_MIXED = 1 };
/* PCB_FP64: every step in double precision.
 * PCB_MIXED: the preconditioner (transforms, per-frequency solves, multigrid) runs in FP32; the
 * operator product of the inner MINRES iterations runs in two-word FP32 arithmetic (theta = 1 and
 * a constant coefficient; see pcb_lanczos_product); true residuals, the other products, inner
 * products, orthogonalisation and vector updates stay FP64, and an FP64 iterative-refinement
 * loop restores the requested true relative residual. */

enum pcb_operator { PCB_OP_A = 0, PCB_OP_AHAT = 1 };
/* PCB_OP_A    : A     = [[alpha I, T^T], [T, -alpha I]]   (Eq. matrix_A; symmetric)
 * PCB_OP_AHAT : A_hat = [[T, -alpha I], [alpha I, T^T]]   (Eq. matrix_A_hat)
 * T = B_n (x) I_m + tau I_n (x) K (Eq. matrix_T), B_n = B^(1) (B^(2))^{-1}. */

enum pcb_precond {
  PCB_PREC_NONE = 0,
  PCB_PREC_ABS_PS = 1,  /* |P_S|^{-1}  (Eq. matrix_P), MINRES route; needs a(x) = 1            */
  PCB_PREC_PS = 2,      /* P_S^{-1}    (Eq. matrix_P_GMRES); a(x) = 1 pointwise, else multigrid */
  PCB_PREC_PMS = 3      /* P_MS^{-1}   (Eq. matrix_P_MS); a(x) = 1 exact, else multigrid        */
};

enum pcb_method { PCB_METHOD_AUTO = 0, PCB_MINRES = 1, PCB_GMRES = 2, PCB_FGMRES = 3 };
/* AUTO: MINRES with |P_S| (theta = 1, a = 1) or P_MS (a variable, theta = 1); GMRES with P_S
 * (theta < 1, a = 1, and every Neumann problem); FGMRES with multigrid P_S (a variable,
 * theta < 1). */

enum pcb_bc { PCB_BC_DIRICHLET = 0, PCB_BC_NEUMANN = 1 };
/* DIRICHLET (Sec. 1, Examples 1-2): N interior nodes per side, h = 1/(N+1), zero boundary values.
 * NEUMANN (Sec. 4, Example 3, homogeneous Neumann): N nodes per side including the boundary,
 *   x_i = i h, h = 1/(N-1); K = a (4 u - sum of neighbours)/h^2 with the missing neighbour of a
 *   boundary node mirrored across it.  This K is not symmetric and enters A and P_S as printed
 *   (K in both diagonal blocks), so A is not symmetric: GMRES with P_S only.  The spatial
 *   transform is the DCT-I of order N-1 in place of the DST-I. */

/* ---- problem --------------------------------------------------------------------------- */
typedef struct pcb_problem pcb_problem;   /* opaque, owned by the library */

typedef struct {
  int N;                  /* points per side.  Dirichlet: interior points, N+1 = 2^a * 3^b      */
                          /* (DST radices), N <= 511; variable a(x) needs N = 2^k - 1          */
                          /* (multigrid).  Neumann: all nodes, N-1 = 2^a * 3^b, 3 <= N <= 513  */
  int n;                  /* time steps; a power of two, 2 <= n <= 1024 (<= 512 with variable a)*/
  double theta;           /* 1/2 <= theta <= 1                                                 */
  double T;               /* horizon, > 0                                                      */
  double gamma;           /* regularisation, > 0                                               */
  double zeta;            /* omega = exp(i zeta), Sec. 2 (pi: the paper's skew-circulant).      */
                          /* Any zeta runs the pipelined FP32 kernels for n <= 512 (pi also for */
                          /* n = 1024); variable a(x) needs zeta = pi                           */
  const double* a_edges;  /* host; NULL => a(x) = 1; else 2*N*(N+1) values of a at cell-edge   */
                          /* midpoints: first ax[j][e] (N rows of N+1; x1-edge between nodes   */
                          /* e and e+1 of row j+1), then ay[e][i] (N+1 rows of N)              */
  int precision;          /* pcb_precision                                                     */
  int mg_cycles;          /* V-cycles per shifted solve when a(x) varies; <= 0 => 2            */
  void* stream;           /* cudaStream_t the problem's work is queued on; NULL = default      */
  int bc;                 /* pcb_bc; 0 = Dirichlet                                             */
  double a_const;         /* constant a(x) when a_edges is NULL; <= 0 => 1.  Neumann requires   */
                          /* a_edges = NULL                                                    */
  int fem;                /* 0: finite differences (M = I, K = -L).  1: bilinear (Q1) finite     */
                          /* elements on the same grid (Sec. 1: M the mass, K the stiffness      */
                          /* matrix; the system carries M^{-1/2} K M^{-1/2}); Dirichlet, constant */
                          /* a, single problems (not batches or the server), y0 = 0              */
  int multigrid;          /* 1: solve the shifted spatial systems of P_S^{-1} / P_MS^{-1} with     */
                          /* mg_cycles multigrid V-cycles also for a constant coefficient (the    */
                          /* route the paper takes for Example 3's Neumann grid, Sec. 4):         */
                          /* Dirichlet N = 2^k - 1, Neumann N = 2^k + 1 >= 5; zeta = pi, n <= 512 */
} pcb_desc;

/* Validate the descriptor, compute the spectral tables (Sec. 3.5: lambda_k(S_n), the eigenvalues
 * of -L, twiddle tables) and allocate the workspaces.  Errors: INVALID_ARG, UNSUPPORTED
 * (N+1 not 2^a 3^b, n not a power of two, N > 511, variable a with N != 2^k - 1 or zeta != pi;
 * Neumann with N-1 not 2^a 3^b, N < 3 or N > 513, or with a_edges), OUT_OF_MEMORY, CUDA.  A zero eigenvalue of S^(2) (Remark 1, e.g. theta = 1/2, zeta = 0) is
 * replaced by 1.  For zeta other than 0 and pi the preconditioners are complex; applied to real
 * vectors they return the real part (a real symmetric positive definite operator for |P_S|). */
int pcb_create(const pcb_desc* desc, pcb_problem** out);
void pcb_destroy(pcb_problem* p);
const char* pcb_status_str(int status);

/* Number of unknowns 2*m*n and the device bytes the problem's workspaces hold. */
long long pcb_unknowns(const pcb_problem* p);
long long pcb_workspace_bytes(const pcb_problem* p);

/* Right-hand side (Sec. 1, vectors f~, g~, then Eq. main_system / main_system_nonsym):
 * g_dev, f_dev: (n+1)*m samples at t_k = k*tau; y0_dev: m values or NULL (= 0).
 * Writes b_dev (2*m*n) for operator `op`.  Finite elements (fem = 1): f~, g~ carry the mass matrix
 * and b the factor M^{-1/2} of Eq. (main_system); y0_dev must be NULL (else UNSUPPORTED). */
int pcb_assemble_rhs(pcb_problem* p, int op, const double* g_dev, const double* f_dev,
                     const double* y0_dev, double* b_dev);

/* y = A x or y = A_hat x (op = pcb_operator); x_dev and y_dev must not overlap. */
int pcb_matvec(pcb_problem* p, int op, const double* x_dev, double* y_dev);

/* One Lanczos step of preconditioned MINRES (Paige and Saunders; the Krylov solver of Sec. 3/4
 * for the symmetric system of Eq. matrix_A): with A the all-at-once operator,
 *     out  = A y / beta - (beta / oldb) r1      (the r1 term is left out when oldb == 0)
 *     *dot = y . out / beta                      (host, FP64)
 * which is the product a MINRES iteration of pcb_solve computes before its scalar step.
 * precision PCB_FP64: FP64 arithmetic (the form of FP64 solves and of true residuals);
 * PCB_MIXED: the two-word FP32 arithmetic of the inner iterations of a mixed-precision solve
 * (inputs split into two FP32 words, 47 of their 53 significand bits; each value accurate to
 * about 2^-46 of the magnitudes of its terms), used for theta = 1 and a constant coefficient;
 * other instances compute in FP64 either way.  y_dev, r1_dev, out_dev: device, 2*m*n each,
 * out_dev distinct from both inputs; r1_dev may be NULL when oldb == 0.  beta > 0 and oldb >= 0,
 * both finite, else INVALID_ARG.  The two-word path splits y relative to the binade of beta and r1
 * relative to that of oldb, so the scale of the right-hand side does not matter; the output and
 * its terms must lie in the FP32 range (as they do in a MINRES iteration, where they do not
 * depend on that scale); a value beyond it comes out non-finite, which the solver reports.
 * Overwrites the problem's MINRES scalars (a later pcb_solve resets them); blocks until *dot is
 * read.  Finite-element problems compute in FP64 whatever
 * the precision. */
int pcb_lanczos_product(pcb_problem* p, int precision, const double* y_dev, const double* r1_dev, double beta,
                        double oldb, double* out_dev, double* dot);

/* y = P^{-1} x for kind = pcb_precond, computed in `precision` (pcb_precision).
 * x_dev and y_dev may be the same buffer.  Uses the problem's scratch workspace, so calls on
 * one problem are serialised by its stream.  UNSUPPORTED: |P_S| with variable a(x); |P_S| and
 * P_MS for Neumann problems (MINRES preconditioners; the Neumann A is not symmetric). */
int pcb_precond_apply(pcb_problem* p, int kind, int precision, const double* x_dev, double* y_dev);

/* ---- autotuning of the preconditioner's kernel shapes ------------------------------------ */
/* The transforms of Sec. 3.5 (steps 1 and 3) can run in several kernel configurations: the
 * pipelined FP32 kernels or the tile kernels for the spatial and the time passes (and, for n = 512,
 * with or without handing the time pass contiguous time lines, and with 2, 3 or 4 resident blocks
 * per SM for that time pass), and for the tile kernels several register-FFT radices (values per
 * lane) and tile sizes.  pcb_autotune times `reps` applications
 * of preconditioner `kind` (PCB_PREC_NONE: the problem's default) in the problem's precision under
 * each configuration that fits the problem's shape, keeps the fastest for this problem, and records
 * it for the device and shape (N, n, boundary condition, zeta = pi or not, precision): problems
 * and server requests of that shape created afterwards start with it.  Every configuration computes
 * the same operator: each candidate's result is compared with the default configuration's on the
 * same input, and one that differs by more than the precision's rounding (relative max-norm 1e-5
 * in FP32, 1e-12 in FP64) is rejected instead of timed.  Blocks while it runs; uses a temporary
 * device buffer of three vectors.  Constant coefficient only (UNSUPPORTED with variable a(x)).
 * Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA. */
typedef struct {
  int candidates;          /* configurations timed                                               */
  int rejected;            /* configurations whose result did not match the default's            */
  int chosen;              /* index of the winner among them (0: the default configuration)      */
  double default_ms;       /* mean apply time of the default configuration                       */
  double best_ms;          /* mean apply time of the winner                                      */
  int pipelined_dst;       /* winner: pipelined spatial passes (1) or tile kernels (0)            */
  int pipelined_time;      /* winner: pipelined time pass (1) or tile kernel (0)                  */
  int time_major_handoff;  /* winner: the n = 512 spatial pass writes contiguous time lines       */
  int dst_lanes;           /* lanes per spatial line of the tile kernels (values per lane = M/lanes)*/
  int time_lanes;          /* lanes per time line of the tile kernels                            */
  double tile_scale;       /* tile size of the tile kernels relative to the default (0.5, 1, 2)   */
  int time512_blocks;      /* winner: resident blocks per SM of the n = 512 time pass (2, 3 or 4) */
} pcb_tune_info;
int pcb_autotune(pcb_problem* p, int kind, int reps, pcb_tune_info* info);

/* Run this problem (only; nothing is recorded for its shape) in configuration `candidate` of the
 * list pcb_autotune times for its shape and precision, in that list's order (0: the default
 * configuration), without timing it; candidate < 0 changes nothing.  `info` (may be NULL) receives
 * the configuration the problem then runs, with `candidates` the length of the list, `chosen` =
 * candidate and zero times.  Lets a caller pin a configuration, and a test compare every one with
 * the oracle.  Errors: INVALID_ARG (candidate past the list), UNSUPPORTED (variable a(x)), CUDA. */
int pcb_tune_select(pcb_problem* p, int candidate, pcb_tune_info* info);

/* Undo the symmetrising change of variables of Eq. (main_system):
 * y = (B2^{-1} (x) M^{-1/2}) x_half0 / sqrt(gamma), p = (B2^{-T} (x) M^{-1/2}) x_half1; each m*n
 * (M = I for finite differences). */
int pcb_recover(pcb_problem* p, const double* x_dev, double* y_dev, double* p_dev);

/* ---- solve ----------------------------------------------------------------------------- */
typedef struct {
  int method;             /* pcb_method                                                        */
  int precond;            /* pcb_precond; PCB_PREC_NONE with method AUTO => the method's default*/
  double tol;             /* target true relative residual ||b - op x||_2/||b||_2 (FP64); <=0 => 1e-8 */
  int maxit;              /* total Krylov iterations; <= 0 => 500                              */
  int restart;            /* GMRES/FGMRES restart length; <= 0 => 30 (max 64)                  */
  int max_refinements;    /* mixed precision: outer refinement sweeps; <= 0 => 10              */
  int fixed_iterations;   /* > 0: run exactly this many iterations (comparison runs)           */
  int profile;            /* != 0: time every preconditioner apply and matvec with CUDA events  */
                          /* recorded on the problem's stream (fills the *_ms fields of info)   */
  double inner_floor;     /* mixed precision: an inner solve stops once its residual estimate is */
                          /* below max(tol*||b||/||r||, inner_floor); <= 0 => no floor          */
  int no_graphs;          /* != 0: launch every iteration's kernels directly.  0: capture one    */
                          /* MINRES iteration, or one FGMRES Arnoldi step per index, into CUDA   */
                          /* graphs once per solve setting and replay them (not with            */
                          /* profile != 0 or a variable a(x))                                   */
} pcb_solve_opts;

typedef struct {
  int status;             /* same as the return value                                          */
  int method;             /* method used                                                       */
  int precond;            /* preconditioner used                                               */
  int iterations;         /* Krylov iterations summed over refinement sweeps                    */
  int refinements;        /* refinement sweeps (1 for FP64)                                    */
  double relres;          /* true FP64 relative residual at exit                                */
  double seconds;         /* wall time of the call                                             */
  long long launches;     /* CUDA kernel launches the call issued                              */
  int precond_applies;    /* preconditioner applications                                       */
  double precond_ms;      /* profile != 0: summed device time of the applications              */
  int matvecs;            /* operator products (Krylov and true-residual)                      */
  double matvec_ms;       /* profile != 0: summed device time of the products                  */
  int matvecs_inner;      /* products of the inner MINRES iterations of a mixed-precision solve */
                          /* (two-word FP32 arithmetic where the problem allows it)            */
  double matvec_inner_ms; /* profile != 0: their summed device time (included in matvec_ms)    */
} pcb_solve_info;

/* Solve op x = b from a zero initial guess, op = A for MINRES and A_hat for (F)GMRES.
 * b_dev, x_dev: device, 2*m*n each; info may be NULL.  Blocks until the solve ends.
 * Neumann problems take GMRES with P_S (AUTO); MINRES or another preconditioner is UNSUPPORTED. */
int pcb_solve(pcb_problem* p, const pcb_solve_opts* opts, const double* b_dev, double* x_dev,
              pcb_solve_info* info);

/* Same solve through host buffers: copies b_host to the device, solves, copies x back
 * (device staging buffers are allocated on the first call and kept until pcb_destroy).
 * Page-locked host buffers are read and written by a copy kernel over the CPU-GPU link;
 * pageable ones go through cudaMemcpyAsync.  info->launches counts the copy kernels. */
int pcb_solve_host(pcb_problem* p, const pcb_solve_opts* opts, const double* b_host,
                   double* x_host, pcb_solve_info* info);

/* ---- allocation-free preconditioner apply ---------------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers that cannot allocate
 * device memory (code running where the device allocator is off limits, memory-capped or
 * pre-partitioned processes, or plain C callers that want no handle to create and destroy).
 * It computes y = P^{-1} x exactly like pcb_precond_apply, for a(x) = 1, without any
 * cudaMalloc/cudaFree: the problem description, the spectral tables and the transform scratch
 * live in one file-scope device array of PCB_NOALLOC_ARENA_BYTES that every GPU loading the
 * library holds until the process exits.
 *   desc       : as for pcb_create (a_edges must be NULL; desc->precision is ignored in favour of
 *                `precision`); the apply is queued on desc->stream.  The call first copies its
 *                descriptor and spectral tables (at most 160 KB) from host memory into the
 *                array with cudaMemcpyAsync, so the host may wait for earlier work on the
 *                stream, and no call may be made while that stream is being captured.
 *   x_dev/y_dev: caller-owned device buffers of 2*m*n FP64 values; they may be the same buffer.
 * Errors: INVALID_ARG, UNSUPPORTED (as pcb_create, or variable a(x)), TOO_LARGE when the tables
 * plus 2*m*n scratch values (4 bytes each for PCB_MIXED, 8 for PCB_FP64) exceed the arena (about
 * 16.7 million unknowns mixed, 8.3 million FP64), CUDA.
 * Every call shares the one array: calls whose GPU work overlaps (different streams, or several
 * host threads) race on it; serialise them, e.g. on one stream.  The scratch needs no clearing
 * between calls (each apply overwrites all of it).  The first call on a device also looks up the
 * array's device address and uploads the transforms' constant tables (synchronous copies). */
#define PCB_NOALLOC_ARENA_BYTES (64ull * 1024ull * 1024ull)
int pcb_precond_apply_noalloc(const pcb_desc* desc, int kind, int precision, const double* x_dev,
                              double* y_dev);

/* ---- device figures -------------------------------------------------------------------- */
/* The paper has no counterpart: a diagnostic for the rooflines of the FP64 steps (the product,
 * the residual and the Krylov updates, which this GPU's narrow FP64 pipe bounds before its memory).
 * Measures the device's FP64 fused multiply-add and add instruction rates (instructions per second;
 * one FMA is two flops) with register-only kernels queued on `stream` (NULL = default); blocks until
 * they finish (about a tenth of a second).  Errors: INVALID_ARG, OUT_OF_MEMORY, CUDA. */
int pcb_measure_fp64_rates(void* stream, double* fma_per_s, double* add_per_s);

/* ---- batches --------------------------------------------------------------------------- */
/* Solve `count` independent problems (uneven N, n, theta, gamma allowed; all with the same
 * precision) with shared kernel launches: every launch of an iteration covers all unfinished
 * problems.  opts applies to each.  Blocks until all finish. */
int pcb_batch_solve(pcb_problem* const* problems, int count, const pcb_solve_opts* opts,
                    const double* const* b_dev, double* const* x_dev, pcb_solve_info* infos);

/* ---- continuous-batching server -------------------------------------------------------- */
/* Requests (independent control solves of any supported size) are queued with pcb_server_submit
 * and advanced by pcb_server_step.  Each step retires finished requests (their solution is copied
 * to the caller's host buffer), admits queued requests, and advances every admitted request by one
 * Krylov iteration (or one refinement transition) in launches shared by all admitted requests of
 * the same method.  Krylov state stays on the device from admission to retirement.  Each request
 * runs the same rounds as pcb_batch_solve, so its result does not depend on which other requests
 * share the launches (reductions are per request and in a fixed order).
 * Memory: pcb_server_create reserves the budget once (at most the device's free memory less 2 GiB);
 * an admitted request's workspace is one block of that reservation (its tables, preconditioner
 * scratch, Krylov vectors and device copies of b and x), returned when it retires, so admission and
 * retirement allocate and free no device memory.
 * Admission: queued requests are considered in arrival order, and each one that finds a free slot of
 * its method and a block of the reservation is admitted, so a large request that does not fit yet
 * does not hold back the small ones behind it; once the oldest queued request has been passed over
 * for 64 steps, nothing else is admitted until it is. */
typedef struct pcb_server pcb_server;

typedef struct {
  long long budget_bytes; /* device bytes reserved for the admitted requests' workspaces (> 0)    */
  int max_slots;          /* concurrent requests per method (1..256)                              */
  int precision;          /* pcb_precision of every request                                       */
  double tol;             /* target true relative residual; <= 0 => 1e-8                          */
  int maxit;              /* Krylov iterations per request; <= 0 => 500                           */
  int restart;            /* GMRES restart length; <= 0 => 16                                     */
  void* stream;           /* cudaStream_t all server work is queued on                           */
} pcb_server_opts;

typedef struct {
  long long tag;          /* caller's tag from pcb_server_submit                                  */
  int status;             /* PCB_OK, PCB_NOT_CONVERGED or a negative error                         */
  int iterations;         /* Krylov iterations                                                     */
  int refinements;        /* refinement rounds                                                     */
  double relres;          /* true FP64 relative residual                                          */
} pcb_server_done;

int pcb_server_create(const pcb_server_opts* opts, pcb_server** out);
void pcb_server_destroy(pcb_server* s);
/* Queue one request.  desc: as for pcb_create (a_edges must be NULL; precision and stream come from
 * the server).  op_rhs_host: the 2*m*n right-hand side for the method pcb_create would pick (A for
 * theta = 1, A_hat otherwise), host memory read when the request is admitted; x_host: 2*m*n host
 * values written when it retires.  Both must stay valid until the request is reported done.
 * Errors: INVALID_ARG, UNSUPPORTED, TOO_LARGE (the request's workspace alone exceeds the
 * reservation). */
int pcb_server_submit(pcb_server* s, const pcb_desc* desc, const double* rhs_host, double* x_host, long long tag);
/* One scheduling step (blocks while it runs).  Up to max_done retired requests are written to done[];
 * *n_done, *n_active and *n_queued report the counts after the step. */
int pcb_server_step(pcb_server* s, pcb_server_done* done, int max_done, int* n_done, int* n_active, int* n_queued);

#ifdef __cplusplus
}
#endif
#endif /* PCB_H */
