/*
 * hdgmg.h -- C ABI of a GB300 (sm_103a) library for the hybridized DG trace
 * system and its DtN-based geometric multigrid (Wildey, Muralikrishnan,
 * Bui-Thanh, "Unified geometric multigrid algorithm for hybridized high-order
 * finite element methods", arXiv:1811.09909).
 *
 * Problem (Sec. 2, eq. primal_elliptic / mixed_elliptic, K = kappa I):
 *     -div(kappa grad u) = f in Omega = [x0,x1] x [y0,y1],  u = g_D on dOmega,
 * discretised by HDG (eqs. HDG_local1, HDG_local2, HDG_flux, conservation)
 * on a uniform n x n mesh of rectangles, volume space Q_p (tensor Lagrange at
 * the (p+1)^2 Gauss-Legendre nodes), trace space P_p per edge in the
 * L2-orthonormal Legendre basis.  Static condensation gives the trace system
 * A lambda = g of Sec. 3 (eq. trace_linear_system), solved by a Krylov method
 * preconditioned with the V-cycle of Algorithm 1 (p-coarsening to P_1, Sec.
 * 3.1.1, then 2x2 agglomeration, Sec. 3.1.2, transfers eqs. n_1_Ik / n_1_Qk,
 * Galerkin coarse operators eq. coarse, edge block-Jacobi smoothing and the
 * local correction eq. localCorrection); u and q are then recovered element
 * by element.
 *
 * Conventions shared by every call
 * --------------------------------
 *  element   e = j*n + i           (i along x, j along y)
 *  edges     vertical edge at x_i, row j:   j*(n+1) + i        (i = 0..n)
 *            horizontal edge at y_j, col i: n*(n+1) + j*n + i  (j = 0..n)
 *            n_edges = 2 n (n+1); edges with i in {0,n} (vertical) or j in
 *            {0,n} (horizontal) are Dirichlet edges.
 *  traces    [mode][edge], mode k = 0..p of psi_k = sqrt((2k+1)/|e|) P_k(s),
 *            s running along +x on horizontal and +y on vertical edges.
 *  volume    [node][e], node (a,b) -> b*(p+1)+a at the Gauss-Legendre points
 *            (a along x).  Flux q: [2][node][e], component x first.
 *  q         is the flux q = -kappa grad u (the paper writes u for the flux
 *            and q for the scalar; this interface uses the HDG convention).
 *
 * Memory: every pointer argument marked "device" is a CUDA device pointer on
 * the context's device, owned by the caller, 8-byte aligned; "host" pointers
 * are ordinary host memory owned by the caller.  The library owns the level
 * hierarchy and its workspace (allocated in hdgmg_create, released in
 * hdgmg_destroy).  All work is issued on the stream given to hdgmg_create;
 * calls return after their work is complete on that stream unless stated.
 *
 * Errors: every call returns an hdgmg_status; 0 is success, negative values
 * are errors, and hdgmg_last_error() returns a thread-local message for the
 * last failure.  No call aborts or exits the process.
 */
#ifndef HDGMG_H
#define HDGMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HDGMG_OK = 0,
  HDGMG_EINVAL = -1,      /* invalid argument or unsupported size          */
  HDGMG_ENOMEM = -2,      /* device allocation failed                      */
  HDGMG_ECUDA = -3,       /* CUDA runtime error                            */
  HDGMG_ENOCONV = -4,     /* max_it reached; best iterate and info written */
  HDGMG_EBREAKDOWN = -5,  /* non-positive pivot, NaN/Inf in the iteration  */
  HDGMG_ETIMEOUT = -6     /* a bounded device wait expired                 */
} hdgmg_status;

/* tau = c, tau = c / h_min, tau_e = c kappa_e / h_min (per element) */
enum { HDGMG_TAU_CONST = 0, HDGMG_TAU_OVER_H = 1, HDGMG_TAU_KAPPA_OVER_H = 2 };
enum { HDGMG_LC_NONE = 0, HDGMG_LC_PRE = 1, HDGMG_LC_BOTH = 2 };
enum { HDGMG_KRYLOV_NONE = 0, HDGMG_KRYLOV_CG = 1, HDGMG_KRYLOV_GMRES = 2 };
enum { HDGMG_PREC_FP64 = 0, HDGMG_PREC_FP32 = 1, HDGMG_PREC_FP32_IR = 2, HDGMG_PREC_BF16 = 3 };
enum { HDGMG_PDE_DIFFUSION = 0, HDGMG_PDE_CONVDIFF = 1 };
/* local discretisation (Sec. 2): HDG (eqs. HDG_local1/2, HDG_flux) or one of
 * the hybridized interior penalty schemes of eq. IPG_H, s_f = 1, -1, 0 */
enum { HDGMG_SCHEME_HDG = 0, HDGMG_SCHEME_SIPG = 1, HDGMG_SCHEME_NIPG = 2,
       HDGMG_SCHEME_IIPG = 3 };
/* smoothers of Sec. 4.1 */
enum { HDGMG_SMOOTH_BLOCK_JACOBI = 0, HDGMG_SMOOTH_POINT_JACOBI = 1,
       HDGMG_SMOOTH_CHEBYSHEV = 2, HDGMG_SMOOTH_LU_SGS = 3 };
/* element condensation (Sec. 2): BASIS uses one basis in which every
 * element's volume block kappa G + S0 is (block) diagonal -- for symmetric
 * blocks the eigenbasis of the pencil (G, E), for non-symmetric ones that of
 * B^-1 G with B the block at kappa's geometric mean, checked at every set-up
 * against direct solves at the extreme kappa (1e-11) -- so no element is
 * factored; FACTOR factors each element's volume block (Cholesky / LU) and
 * keeps the factors; AUTO = BASIS where it is accurate, FACTOR otherwise */
enum { HDGMG_CONDENSE_AUTO = 0, HDGMG_CONDENSE_BASIS = 1, HDGMG_CONDENSE_FACTOR = 2 };

typedef struct hdgmg_ctx hdgmg_ctx;   /* opaque, library-owned */

/* Problem statement (Sec. 2).  n must be a multiple of 2^L so that the mesh
 * halves down to opts.coarsest_n; 1 <= p <= 8.
 *
 * pde = HDGMG_PDE_DIFFUSION: -div(kappa grad u) = f (the paper's problem).
 * pde = HDGMG_PDE_CONVDIFF (an extension, not in the paper):
 *   -div(eps grad u) + div(beta u) = f with constant beta = (beta_x, beta_y)
 *   and eps = exp(log_kappa) per element.  The HDG flux is
 *   q.n + (beta.n) lambda + tau_f (u - lambda) with the upwind
 *   tau_f = tau + max(beta.n_f, 0) on each element face.  The trace operator
 *   is non-symmetric (full storage on every level, the restriction built from
 *   A_BI); use krylov = GMRES or NONE (CG is rejected with EINVAL), and the
 *   adjoint entry points reject it.  Zero-initialised fields (older callers)
 *   select diffusion.
 *
 * scheme (diffusion only; EINVAL with CONVDIFF): HDGMG_SCHEME_HDG (default)
 * or the primal hybridized interior penalty schemes of eq. IPG_H,
 *   (kappa grad u, grad w)_K - s_f <u - lambda, kappa grad w.n>_dK
 *     - <kappa grad u.n, w>_dK + <tau (u - lambda), w>_dK = (f, w)_K,
 * flux uhat.n = -kappa grad u.n + tau (u - lambda) (eq. IPDG_flux) in the
 * conservation condition.  SIPG-H (s_f = 1) is symmetric and runs the
 * symmetric path (CG allowed; the adjoint too); NIPG-H (s_f = -1) and
 * IIPG-H (s_f = 0) are non-symmetric and take the same path and limits as
 * CONVDIFF (GMRES or NONE).  The recovered flux is q = -kappa grad u at the
 * volume nodes.  The paper uses tau = (p+1)(p+2)/h_min (TAU_OVER_H with
 * tau_c = (p+1)(p+2)); with a variable kappa, TAU_KAPPA_OVER_H keeps the
 * penalty proportional to kappa_e.  A tau too small for the scheme makes the
 * volume block indefinite: set-up then returns HDGMG_EBREAKDOWN. */
typedef struct {
  int32_t n;              /* elements per side                               */
  int32_t p;              /* polynomial order                                */
  double x0, x1, y0, y1;  /* domain                                          */
  int32_t tau_mode;       /* HDGMG_TAU_* (Sec. 4.1)                          */
  double tau_c;           /* the constant c                                  */
  int32_t pde;            /* HDGMG_PDE_DIFFUSION or HDGMG_PDE_CONVDIFF       */
  double beta_x, beta_y;  /* convection velocity (CONVDIFF only)             */
  int32_t scheme;         /* HDGMG_SCHEME_* (0 = HDG)                        */
} hdgmg_problem;

/* Solver options.  hdgmg_default_opts() fills the documented defaults. */
typedef struct {
  int32_t coarsest_n;     /* agglomerate until n <= coarsest_n (>= 2); 2     */
  int32_t m_fine;         /* smoothing steps m_N on the finest level; 1      */
  int32_t m_growth;       /* m_{k-1} = m_growth * m_k (Sec. 3.3, beta); 2    */
  int32_t m_max;          /* cap on m_k (0 = none); 0                        */
  int32_t local_corr;     /* HDGMG_LC_*: step 3 / steps 3+5 of Alg. 1; BOTH  */
  double omega;           /* block-Jacobi damping (1 = paper, undamped); 1   */
  int32_t krylov;         /* NONE = MG as fixed-point solver, CG (symmetric
                             cycle), GMRES = flexible GMRES(gmres_restart)
                             right-preconditioned by the cycle (the paper's
                             Krylov method, Sec. 4); CG                       */
  int32_t max_it;         /* outer iterations; 200                           */
  double rtol;            /* ||g - A lambda||_2 / ||g||_2 target; 1e-10      */
  int32_t precision;      /* FP64: PCG in FP64 with the FP64 V-cycle.
                             FP32: PCG in FP64 (FP64 operator, residual and
                             dot products) preconditioned by the FP32 V-cycle.
                             FP32_IR: iterative refinement -- FP64 residual of
                             the FP64 operator, inner FP32 PCG with the FP32
                             V-cycle on the normalised residual.
                             BF16: as FP32, but the finest level's V-cycle
                             matvecs read a BF16 copy of the element
                             operators (FP32 accumulation; block-Jacobi
                             blocks and coarse levels from the FP64
                             operator, rounded to FP32); FP64                */
  double inner_rtol;      /* FP32_IR only: inner PCG tolerance per refinement
                             step, in (0,1); 1e-5                             */
  int32_t cluster_tail_n; /* > 0: the P1 levels with n <= this run fused in
                             one thread-block cluster (distributed shared
                             memory); <= 0: not used (the single-block tail
                             and separate launches are faster on GB300); 0   */
  int32_t gmres_restart;  /* GMRES restart length m, 1..256; 30              */
  int32_t smoother;       /* HDGMG_SMOOTH_*, Sec. 4.1: BLOCK_JACOBI (one block
                             per edge, damped by omega), POINT_JACOBI (damped
                             by omega; the paper uses 2/3), CHEBYSHEV
                             (point-Jacobi accelerated on [L/30, L], L the
                             largest eigenvalue of D^-1 A from 30 power
                             iterations at set-up), LU_SGS (one forward and
                             one backward point Gauss-Seidel sweep per step,
                             multicolour edge order: vertical edges of even,
                             odd column, horizontal of even, odd row; then
                             mode).  The fused single-block tail and the
                             fused edge sweeps serve BLOCK_JACOBI only;
                             BLOCK_JACOBI                                    */
  int32_t condensation;   /* HDGMG_CONDENSE_*: AUTO = BASIS where the basis
                             is accurate (always for symmetric blocks), else
                             FACTOR; BASIS when the non-symmetric basis fails
                             its accuracy check: hdgmg_setup returns EINVAL;
                             AUTO                                            */
  int32_t l2_persist_mb;  /* > 0: the Krylov loop graphs mark the finest
                             operator the V-cycle reads (its BF16, FP32 or
                             FP64 copy) as persisting in L2, with a set-aside of
                             this many MiB (capped by the device; the set-aside
                             is a limit of the calling process's context, the
                             persisting lines are reset by hdgmg_destroy); 0:
                             off.  hdgmg_batch_create uses 0 for its contexts.
                             64                                              */
  int32_t pcycle;         /* 1: with BLOCK_JACOBI, the P1 levels of every
                             FP32 V-cycle (from the first P1 level down to
                             the coarsest and back) run as ONE cooperative
                             kernel launch, the steps separated by grid
                             barriers whose waits are bounded (a wait that
                             runs out makes the solve return HDGMG_ETIMEOUT
                             and leaves the context usable); the FP64 cycle
                             stays launched (faster on GB300); 2: the FP64
                             cycle too; 0: separate launches per step plus
                             the single-block tail.  Needs a coarsest level
                             with at most 4096 unknowns; otherwise the
                             launched form runs.  1                         */
  int32_t pcycle_tail_n;  /* pcycle = 1: the levels with n <= this run on
                             one thread block of the launch (block barriers)
                             while the others wait at one grid barrier; 0:
                             every level on the whole grid.  16             */
  int32_t pcg_graph;      /* 1: the PCG loop (krylov = CG, precision FP64,
                             FP32 or BF16) runs as one CUDA graph with a
                             device-side while node; 0: every iteration's
                             kernels are launched from the host, which reads
                             the stop test back after each iteration (same
                             arithmetic; for per-kernel profiling).  1       */
  int32_t rhs_block;      /* > 1: hdgmg_solve with nrhs > 1 solves blocks of
                             up to rhs_block (<= 16) right-hand sides
                             together: FP64 iterative refinement (residual of
                             the FP64 operator per right-hand side) around
                             k simultaneous FP32 PCGs that share every
                             V-cycle, FP32 matvec and vector pass (each
                             level operator is read once for all k).  Needs
                             a symmetric operator, krylov CG, BLOCK_JACOBI
                             and precision FP32 or FP32_IR (EINVAL
                             otherwise); info then describes the last block
                             (iters: inner iterations, rel_res: the worst
                             right-hand side).  0 or 1: one at a time.  0    */
  int32_t pcg_fuse;       /* 1: each FP64 PCG iteration (krylov = CG, one
                             right-hand side) forms the direction update, the
                             FP64 matvec and p.Ap in one kernel and x, r, p in
                             one more (the matvec gathers p + beta z where the
                             elements read it; p.Ap summed element by element,
                             sum_e p_e^T A_e p_e); 0: separate direction,
                             matvec, dot and update kernels.  Same iteration,
                             different summation order.  1                   */
  int32_t matrix_free;    /* 1: the V-cycle applies the finest operator
                             matrix-free in FP32 through the shared
                             eigenbasis, A_e x = kappa K x + tau x -
                             sum_i (kappa P_i + tau Q_i)^T (...) x / s_i
                             (nt^2 + 4 nv nt FMA per element, no stored
                             entries read); the FP64 operator of the Krylov
                             iteration stays stored.  Needs the symmetric
                             basis condensation, p <= 6 and precision FP32
                             or FP32_IR (EINVAL otherwise).  0: stored.  0   */
} hdgmg_opts;

typedef struct {
  int32_t iters;          /* Krylov iterations = V-cycle applications       */
  int32_t converged;      /* 1 if rel_res <= rtol                            */
  double rel_res;         /* ||g - A lambda|| / ||g||, recomputed in FP64    */
  double t_setup_ms;      /* device time of the last hdgmg_setup             */
  double t_solve_ms;      /* device time of the last hdgmg_solve             */
  int32_t n_levels;
  int64_t trace_dofs;     /* interior trace unknowns 2 n (n-1) (p+1)         */
  int64_t kernel_launches; /* kernels run by the last setup + solve (graph
                              nodes counted once per replay)                 */
  int32_t refinements;    /* FP32_IR: outer FP64 refinement steps, else 0    */
  double t_condense_ms;   /* device time of the element condensation kernel
                             in the last hdgmg_setup (CUDA events around it) */
  int32_t condense_threads; /* threads per element the condensation kernel
                             ran with (symmetric blocks: 128 threads shared by
                             the block's elements, i.e. 128 / EPB), and ...   */
  int32_t condense_elements_per_block; /* ... elements per block: picked once
                             per (kernel, p, device) by timing candidate
                             shapes on the first set-up; the result does not
                             depend on them                                   */
  int32_t condense_kind;  /* HDGMG_CONDENSE_BASIS or _FACTOR: what ran      */
} hdgmg_info;

void hdgmg_default_opts(hdgmg_opts* opts);

/* Create a context for one problem: validates sizes, builds the reference
 * element tables on the host and allocates every device buffer of the
 * hierarchy on the current device.  stream: a cudaStream_t (NULL = legacy
 * default stream).  On error *ctx is NULL. */
hdgmg_status hdgmg_create(hdgmg_ctx** ctx, const hdgmg_problem* problem,
                          const hdgmg_opts* opts, void* stream);

/* Set-up (Sec. 2 static condensation; Sec. 3.1-3.2 hierarchy):
 *   log_kappa  device, [n*n] FP64, per-element log-diffusivity.
 * Runs element condensation (symmetric volume blocks: in the basis that
 * diagonalises every element's kappa G + tau E, built once at create;
 * non-symmetric ones: local LU), the edge block-Jacobi inverses,
 * p-coarsening, every 2x2 agglomeration level and the dense factorisation of
 * the coarsest operator.  EBREAKDOWN if a volume block is not positive
 * definite / a local pivot is not positive (e.g. kappa NaN). */
hdgmg_status hdgmg_setup(hdgmg_ctx* ctx, const double* log_kappa);

/* Solve (Sec. 2-3) for nrhs right-hand sides, one after another:
 *   f       device, [nrhs][(p+1)^2][n*n] FP64 forcing at the Gauss nodes
 *   g_D     device, [nrhs][p+1][n_edges] FP64 Dirichlet trace coefficients
 *           (entries on interior edges are ignored), or NULL for g_D = 0
 *   lambda  device, [nrhs][p+1][n_edges] FP64 out (boundary entries = g_D)
 *   u       device, [nrhs][(p+1)^2][n*n] FP64 out, or NULL
 *   q       device, [nrhs][2][(p+1)^2][n*n] FP64 out, or NULL
 *   info    host, out (may be NULL); describes the last right-hand side.
 * Requires a prior hdgmg_setup.  ENOCONV still writes the last iterate.
 * nrhs = 0 does nothing and returns OK (the array pointers may then be
 * NULL). */
hdgmg_status hdgmg_solve(hdgmg_ctx* ctx, int32_t nrhs, const double* f,
                         const double* g_D, double* lambda, double* u,
                         double* q, hdgmg_info* info);

/* End-to-end call on HOST buffers: copies log_kappa, f, g_D to the device,
 * runs hdgmg_setup and hdgmg_solve for one right-hand side, copies lambda,
 * u, q back.  Same layouts as above; every pointer is host memory (pinned
 * memory gives asynchronous copies); g_D may be NULL. */
hdgmg_status hdgmg_run_host(hdgmg_ctx* ctx, const double* log_kappa,
                            const double* f, const double* g_D,
                            double* lambda, double* u, double* q,
                            hdgmg_info* info);

/* ---- adjoint (gradient with respect to log kappa and f) ----------------- */

/* Gradient of the misfit
 *   J = 1/2 sum_e (u_e - u_obs,e)^T M (u_e - u_obs,e)
 * (M: the Gauss-node volume mass matrix, i.e. the L2 norm evaluated by
 * quadrature on the nodal values) with respect to the per-element
 * log-diffusivity m_e = log kappa_e given to the last hdgmg_setup and to the
 * nodal forcing f.  Runs the forward solve, then one solve of the trace
 * system with right-hand side M (u - u_obs) and homogeneous Dirichlet data
 * (A is symmetric, so the transposed solve is the same multigrid solve),
 * its local recovery, and the per-element contraction
 *   dJ/dm_e = -kappa_e [ w^T (G u - H lambda) + mu^T (K lambda - H^T u) ],
 *   dJ/df_e = M w,
 * with (lambda, u) the forward and (mu, w) the adjoint trace and volume
 * fields (G = sum_d B_d M^-1 B_d^T, H = sum_d B_d M^-1 C_d,
 * K = sum_d C_d^T M^-1 C_d: the q-eliminated HDG blocks of Sec. 2).
 *   f, g_D    device, as in hdgmg_solve (one right-hand side; g_D may be NULL)
 *   u_obs     device, [(p+1)^2][n*n] FP64
 *   J         host, out (may be NULL)
 *   dJ_dlogk  device, [n*n] FP64 out (may be NULL)
 *   dJ_df     device, [(p+1)^2][n*n] FP64 out (may be NULL)
 *   info      host, out (may be NULL): the adjoint solve.
 * The element data of the set-up are reused (kept in memory). */
hdgmg_status hdgmg_gradient(hdgmg_ctx* ctx, const double* f, const double* g_D,
                            const double* u_obs, double* J, double* dJ_dlogk,
                            double* dJ_df, hdgmg_info* info);

/* Adjoint of one solve for a general functional L(u): given the forward
 * trace lambda and volume field u of the last set-up (device, layouts of
 * hdgmg_solve, one right-hand side) and the nodal sensitivity g_u = dL/du
 * (device, [(p+1)^2][n*n]), writes dL/dlog kappa [n*n] and dL/df
 * [(p+1)^2][n*n] (device, either may be NULL).  Used by the torch.autograd
 * binding. */
hdgmg_status hdgmg_adjoint(hdgmg_ctx* ctx, const double* lambda, const double* u,
                           const double* g_u, double* dL_dlogk, double* dL_df,
                           hdgmg_info* info);

/* ---- batching: many independent problems on one GPU ------------------- */

typedef struct hdgmg_batch hdgmg_batch;   /* opaque, library-owned */

/* Create a batch of nprob independent problems (each its own n, p, domain
 * and tau; one set of options for all).  Every problem gets its own context
 * and CUDA stream; nthreads host threads (<= 0: 8) drive them so that the
 * problems run concurrently on the device.  Batch calls are ordered after
 * the work already queued on `stream` and the work they queue is awaited
 * by `stream` through events.  (Batching of independent problems and
 * right-hand sides is not in the paper; every problem is the method of the
 * single-problem entry points.) */
hdgmg_status hdgmg_batch_create(hdgmg_batch** batch, int32_t nprob,
                                const hdgmg_problem* problems,
                                const hdgmg_opts* opts, int32_t nthreads,
                                void* stream);

/* Set-up of every problem: log_kappa is a HOST array of nprob device
 * pointers, each as in hdgmg_setup. */
hdgmg_status hdgmg_batch_setup(hdgmg_batch* batch,
                               const double* const* log_kappa);

/* Solve nrhs right-hand sides of every problem: f, g_D, lambda, u, q are HOST
 * arrays of nprob device pointers laid out as in hdgmg_solve (g_D, u, q and
 * their entries may be NULL); infos: host array of nprob (or NULL).  Returns
 * the first failure in problem order (ENOCONV only if nothing worse). */
hdgmg_status hdgmg_batch_solve(hdgmg_batch* batch, int32_t nrhs,
                               const double* const* f, const double* const* g_D,
                               double* const* lambda, double* const* u,
                               double* const* q, hdgmg_info* infos);

/* The context of problem i (owned by the batch) for the inspection calls. */
hdgmg_status hdgmg_batch_context(hdgmg_batch* batch, int32_t i, hdgmg_ctx** ctx);

void hdgmg_batch_destroy(hdgmg_batch* batch);

/* ---- inspection entry points (used by the parity tests) ---------------- */

/* Number of levels (finest = 0) and the shape of level k: macro-elements per
 * side *n and trace modes per edge *nd (p+1 on level 0, 2 below). */
hdgmg_status hdgmg_num_levels(hdgmg_ctx* ctx, int32_t* n_levels);
hdgmg_status hdgmg_level_shape(hdgmg_ctx* ctx, int32_t level, int32_t* n,
                               int32_t* nd);

/* Copy the per-element operators of level k (Sec. 3: A_e on level 0, the
 * Galerkin macro-element operators of eqs. ANm1 / Akm1 below) as full
 * matrices: out device, [4nd][4nd][n*n] FP64, local order (edge, mode) with
 * edges left, right, bottom, top.  Levels below 0 are held in the V-cycle
 * precision and widened to FP64. */
hdgmg_status hdgmg_copy_element_matrices(hdgmg_ctx* ctx, int32_t level,
                                         double* out);

/* y = A_k x on level k (eq. trace_partition's A_k restricted to interior
 * edges): x, y device, [nd][n_edges(level)] FP64; Dirichlet entries of x are
 * treated as zero and those of y are set to zero.  Level 0 uses the FP64
 * operator; other levels the V-cycle precision. */
hdgmg_status hdgmg_apply_operator(hdgmg_ctx* ctx, int32_t level,
                                  const double* x, double* y);

/* Same result as hdgmg_apply_operator, for callers that cannot allocate
 * device memory when they call it: programs whose device memory is owned by
 * another allocator (a caching allocator that has already reserved the free
 * memory, so a cudaMalloc would fail or fragment it), and latency-critical
 * loops that must not call cudaMalloc/cudaFree (both can synchronise the
 * device and take far longer than the operator itself).  The paper has no
 * counterpart; this is an interface convenience.
 *   Instead of cudaMalloc'd temporaries it uses one static device array of
 *   2^20 doubles (8 MiB) that every GPU loading the library reserves until
 *   the process exits.  Levels with more than 2^20 trace values
 *   (nd * n_edges) are rejected with HDGMG_EINVAL.
 *   The first call on a device resolves the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture begins.
 *   All calls share the array: calls whose work overlaps on the GPU (other
 *   streams, other host threads) race on it.  x, y: as in
 *   hdgmg_apply_operator.  Returns after the work is complete on the
 *   context's stream (the call synchronises that stream). */
hdgmg_status hdgmg_apply_operator_noalloc(hdgmg_ctx* ctx, int32_t level,
                                          const double* x, double* y);

/* e = B_N r: one V-cycle of Algorithm 1 on the finest level, in the V-cycle
 * precision; r, e device, [p+1][n_edges] FP64 (Dirichlet entries ignored /
 * zero). */
hdgmg_status hdgmg_apply_vcycle(hdgmg_ctx* ctx, const double* r, double* e);

/* Check of the bounded waits of the persistent V-cycle (opts.pcycle): runs
 * its kernel once on the context's level vectors with every thread block
 * withholding its arrival at the first grid barrier, so that each block's
 * wait runs out after wait_us (1 ... 10^6) microseconds.  Returns
 * HDGMG_ETIMEOUT when the limit works: the kernel returns by itself, the
 * barrier and the flag are reset, and the context stays usable for further
 * solves.  HDGMG_EINVAL when the context does not run the persistent cycle
 * or before hdgmg_setup.  (A test entry point; the paper has no
 * counterpart.) */
hdgmg_status hdgmg_check_cycle_timeout(hdgmg_ctx* ctx, int32_t wait_us);

/* Step trace of the persistent V-cycle (opts.pcycle): applies one V-cycle
 * exactly as hdgmg_apply_vcycle (same r, e), and thread 0 of block 0 of the
 * persistent kernel records, after each barrier, the device's global timer
 * (ns) and the tag of the step the barrier ended.  stamps: host int64 array
 * of 2 * cap entries, written as (time_ns, tag) pairs; *count: pairs
 * written (at most cap, 1 <= cap <= 4096).  tag = level * 16 + kind, level
 * counted from the first P1 level of the persistent cycle, kind: 0 kernel
 * start, 1 first sweep, 2 down sweep, 3 local correction, 4 residual +
 * restriction, 5 residual, 6 restriction, 7 coarsest solve, 8 prolongation,
 * 9 up sweep, 10 end of the block-0 tail, 11 kernel end (block 0).  The
 * steps of the block-0 tail are stamped after its block barriers.
 * HDGMG_EINVAL when the context does not run the persistent cycle.  (A
 * profiling entry point; the paper has no counterpart.) */
hdgmg_status hdgmg_trace_vcycle(hdgmg_ctx* ctx, const double* r, double* e, int64_t* stamps,
                                int32_t cap, int32_t* count);

/* The condensed right-hand side b = sum_e g_e - A lambda_D on interior
 * edges (Sec. 2; Dirichlet data applied strongly): f, g_D as in hdgmg_solve
 * (one right-hand side), b device [p+1][n_edges] FP64 out. */
hdgmg_status hdgmg_condensed_rhs(hdgmg_ctx* ctx, const double* f,
                                 const double* g_D, double* b);

/* Thread-local description of the last error ("" if none). */
const char* hdgmg_last_error(void);

/* Release every device buffer of the context.  NULL is accepted. */
void hdgmg_destroy(hdgmg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* HDGMG_H */
