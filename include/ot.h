/*
 * ot.h -- C ABI of the GB300 interior-point solver for Benamou-Brenier
 * dynamical optimal transport (Facca, Todeschi, Natale, Benzi,
 * arXiv 2209.00315).
 *
 * Discrete problem (Sec. 2 of the paper).  The density rho and the slack s
 * live on a coarse triangle mesh T' (N' cells) at the K interior times
 * t^k = k dt, k = 1..K, dt = 1/(K+1); the potential phi lives on the fine mesh
 * T (N cells, every coarse triangle split into 4 by its edge midpoints) at the
 * K+1 staggered times (t^{k-1} + t^k)/2.  Spatial operators are two-point-flux
 * finite volumes (Sec. 2.1), time operators are staggered differences and
 * averages (Sec. 2.2), and the log barrier relaxes rho .* s = 0 to
 * rho .* s = mu (Sec. 2.4).
 *
 * Mesh: the unit square cut into n x n squares, each split by its diagonal
 * from (i h, j h) to ((i+1) h, (j+1) h) into a lower-right triangle (t = 0,
 * vertices (i,j),(i+1,j),(i+1,j+1)) and an upper-left one (t = 1, vertices
 * (i,j),(i+1,j+1),(i,j+1)).  A triangle's index is t n^2 + j n + i on the
 * coarse mesh and t (2n)^2 + J (2n) + I on the fine mesh, whose squares have
 * side h/2.  Cell points are circumcentres; on the hypotenuses, where two
 * circumcentres coincide, the distance between barycentres is used instead.
 *
 * Arrays: caller-owned, float64, slice-major:
 *   phi  (K+1) x N      rho, s  K x N'      rho_in, rho_f  N'
 * They are device pointers when options.memspace == OT_MEM_DEVICE (the
 * default) and host pointers when it is OT_MEM_HOST.  Work runs on the CUDA
 * stream passed as `cuda_stream` (NULL = the legacy default stream); the
 * functions return after the results are in the caller's arrays.
 *
 * Errors are returned, never aborted; ot_last_error() gives a message for the
 * last failing call on the calling thread.  The library allocates its own
 * device workspace the first time a mesh is used with a given K and
 * precision, caches it in the mesh object and frees it in ot_mesh_destroy().
 * A mesh object may be used by one thread at a time.
 */
#ifndef OT_H
#define OT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OT_OK = 0,
  OT_ERR_INVALID_ARG = 1,       /* bad size, null pointer, unsupported mesh */
  OT_ERR_MASS_MISMATCH = 2,     /* |c'|.rho_in and |c'|.rho_f differ by > 1e-12 relative */
  OT_ERR_NEGATIVE_DENSITY = 3,  /* rho_in or rho_f has a negative entry, or rho/s <= 0 */
  OT_ERR_NOT_CONVERGED = 4,     /* Newton or FGMRES reached its iteration cap */
  OT_ERR_BREAKDOWN = 5,         /* Krylov breakdown or zero step length */
  OT_ERR_NONFINITE = 6,         /* NaN or Inf in an input or a residual */
  OT_ERR_CUDA = 7,              /* a CUDA runtime call failed */
  OT_ERR_OOM = 8                /* device allocation failed */
} ot_status;

typedef enum { OT_MESH_STRUCTURED_SQUARE = 0, OT_MESH_CARTESIAN_CUBE = 1 } ot_mesh_kind;

/* Mesh description.  STRUCTURED_SQUARE: n squares per side; n = 2^a b with
 * b <= 11 (the multigrid hierarchy coarsens while the side is even).
 * CARTESIAN_CUBE: the 3D variant of test 4 (Sec. 4.1): n^3 cubes of side 1/n
 * on [0,1]^3, 1 <= n <= 1024, density and potential on the same grid (J = I),
 * cube (i, j, k) at index (k n + j) n + i; it supports the operator-level calls
 * ot_residual, ot_kkt_apply and ot_cost_dual (every solver entry point returns
 * OT_ERR_INVALID_ARG for it). */
typedef struct {
  int32_t kind;
  int32_t n;
} ot_mesh_desc;

typedef struct ot_mesh ot_mesh;  /* opaque, library-owned */

typedef enum { OT_MEM_DEVICE = 0, OT_MEM_HOST = 1 } ot_memspace;
typedef enum { OT_PREC_FP64 = 0, OT_PREC_MIXED = 1 } ot_precision;
/* Preconditioner of the outer FGMRES (Sec. 4.2-4.3): BB (the default); SIMPLE;
 * or HYBRID: SIMPLE in the barrier stages with mu < simple_mu, BB before them
 * (the switch the paper proposes for small mu, where BB degrades). */
typedef enum { OT_PRECOND_BB = 0, OT_PRECOND_SIMPLE = 1, OT_PRECOND_HYBRID = 2 } ot_precond;

/* Solver options; ot_default_options() fills the values used by the paper. */
typedef struct {
  int32_t memspace;         /* OT_MEM_DEVICE or OT_MEM_HOST */
  int32_t precision;        /* OT_PREC_FP64: FP64 arithmetic throughout (with gs_shadow = 1 the outer
                               FGMRES takes its Gram-Schmidt coefficients from an FP32 copy of the basis
                               and applies them in FP64); OT_PREC_MIXED: the BB preconditioner in FP32 */
  double mu_factor;         /* mu_{l+1} = mu_factor mu_l (0.2) */
  double tau;               /* fraction to the boundary (0.99) */
  double newton_tol;        /* Newton stop: ||F|| <= newton_tol max(1, ||F_stage_start||) (1e-6) */
  double final_newton_tol;  /* the same for the last mu stage; <= 0: newton_tol */
  double eps_out;           /* FGMRES: ||r|| <= eps_out ||(f;g;h)|| (1e-5, Sec. 3.1) */
  double final_eps_out;     /* the same in the last stage; <= 0: eps_out */
  double eps_schur;         /* inner Schur solve relative tolerance (1e-1, Sec. 4.3.3) */
  int32_t fgmres_restart;   /* restart length; 0 (default): automatic = no restart up to fgmres_max_iter,
                               as far as the 2m+1 Krylov vectors fit 64 GiB (96 GiB shared by the streams
                               of a batched call), never below 30; max 800 */
  int32_t fgmres_max_iter;  /* total FGMRES iterations per linear system (400) */
  int32_t schur_max_iter;   /* inner GMRES iterations per preconditioner application */
  int32_t lap_cycles;       /* multigrid V-cycles per time-slice Laplacian solve */
  int32_t smooth_sweeps;    /* pre- and post-smoothing sweeps per level */
  int32_t coarse_sweeps;    /* smoothing sweeps on the coarsest grid */
  int32_t max_newton;       /* Newton steps per mu stage */
  int32_t verbose;          /* 0: silent; 1: one line per stage on stderr; 2: per Newton step */
  int32_t gs_shadow;        /* 1 (default): the outer Gram-Schmidt dot products read an FP32 copy of the
                               FGMRES basis (coefficients applied to the FP64 basis, so the Arnoldi
                               relation stays FP64); 0: every Gram-Schmidt pass in FP64 */
  int32_t graphs;           /* 1 (default): each FGMRES cycle, with the inner Schur solves of its
                               preconditioner applications, runs as one CUDA graph whose loops are
                               conditional (WHILE) nodes driven by device-side convergence tests;
                               0: the same kernels launched one by one, the host reading the
                               convergence state after every Krylov step */
  int32_t precond;          /* ot_precond: OT_PRECOND_BB (default), OT_PRECOND_SIMPLE or OT_PRECOND_HYBRID.
                               SIMPLE runs in FP64 in both precisions: A^ = Diag(A), its Schur complement
                               solved by GMRES to eps_schur (at most schur_max_iter iterations),
                               preconditioned by exact solves of its time-line (tridiagonal) part;
                               it needs K <= 1024 (OT_ERR_INVALID_ARG otherwise) */
  double simple_mu;         /* HYBRID: SIMPLE for the stages with mu < simple_mu (1e-5) */
  int32_t pdl;              /* 1 (default): the solver's kernels use programmatic dependent launch (each
                               may be scheduled while its predecessor's last blocks finish, then waits
                               for its results); 0: plain stream order.  Results are the same */
} ot_options;

#define OT_MAX_STAGES 40

/* Statistics of a solve (the paper's metrics of Sec. 4, per mu stage). */
typedef struct {
  int32_t stages;
  int32_t newton_steps;
  int64_t fgmres_iters;            /* outer FGMRES iterations, all linear systems */
  int64_t inner_iters;             /* inner Schur iterations, all preconditioner calls */
  double final_residual;           /* ||F|| at the end */
  double mu;                       /* last mu */
  double gap;                      /* mu |Omega| K/(K+1) */
  double cost;                     /* discrete kinetic energy C */
  double dual;                     /* discrete dual value D */
  double seconds;                  /* wall time of the call */
  double stage_mu[OT_MAX_STAGES];
  int32_t stage_newton[OT_MAX_STAGES];
  int64_t stage_outer[OT_MAX_STAGES];
  int64_t stage_inner[OT_MAX_STAGES];
  double stage_seconds[OT_MAX_STAGES];
  double stage_residual[OT_MAX_STAGES];
} ot_stats;

/* Fill `opt` with the defaults above. */
void ot_default_options(ot_options* opt);

/* Create a mesh (Sec. 2.1: coarse mesh for rho and s, its 4-split for phi).
 * Returns OT_ERR_INVALID_ARG for an unsupported description. */
ot_status ot_mesh_create(const ot_mesh_desc* desc, ot_mesh** out);

/* Free a mesh and every workspace cached in it.  NULL is ignored. */
void ot_mesh_destroy(ot_mesh* mesh);

/* Sizes of a mesh; coarse_areas (nullable, host, N') receives |c'|. */
ot_status ot_mesh_info(const ot_mesh* mesh, int64_t* n_coarse, int64_t* n_fine, int64_t* n_edges_fine,
                       double* coarse_areas);

/* Interior-point solve (Sec. 2.4, 3, 4.3).  mu-continuation from mu0 with
 * mu <- mu_factor mu until mu |Omega| K/(K+1) <= tol; each stage runs inexact
 * Newton steps whose linear systems are solved by FGMRES preconditioned with
 * the BB approximation of the Schur complement (Sec. 4.3).
 *   rho_in, rho_f  N' cell averages, >= 0, equal masses (Sec. 2.2)
 *   rho, s         out, K x N';  phi out, (K+1) x N, gauge: zero M-weighted space-time mean
 *   cost           out (nullable): C = dt sum_k 1/2 sum_e |e||w| rho~^k_e (grad phi^k)_e^2
 *   stats          out (nullable)
 * With warm_start != 0 the incoming rho, phi, s are used as the initial point
 * (rho, s > 0); otherwise rho^k interpolates rho_in, rho_f linearly, phi = 0,
 * s = mu0/rho. */
ot_status ot_ipm_solve(ot_mesh* mesh, const double* rho_in, const double* rho_f, int32_t K, double mu0,
                       double tol, const ot_options* opt, int32_t warm_start, double* rho, double* phi,
                       double* s, double* cost, ot_stats* stats, void* cuda_stream);

/* Batched interior-point solves of n_prob independent problems of uneven size
 * (the paper's method applied to each; the batching itself has no counterpart
 * in the paper).  Problem p is ot_ipm_solve(meshes[p], rho_in[p], rho_f[p],
 * K[p], mu0, tol, opt, no warm start, rho[p], phi[p], s[p], cost + p,
 * stats + p); all arrays follow opt->memspace, as in ot_ipm_solve.  The
 * problems run concurrently on n_streams (1..64) non-blocking CUDA streams of
 * the current device, each driven by its own host thread with its own
 * workspaces (largest problems first); the call returns when all are done.
 *   cost, stats, status  nullable arrays of n_prob; status[p] = problem p's code
 * Returns OT_OK, or the code of the first failed problem (the others still run
 * to completion).  Kernel timing (ot_kernel_timing_enable) does not see these
 * solves; the launch counter does.  The caller's meshes must stay alive and
 * must not be used concurrently by other calls. */
ot_status ot_ipm_solve_batched(int32_t n_prob, ot_mesh* const* meshes, const int32_t* K, const double* const* rho_in,
                               const double* const* rho_f, double mu0, double tol, const ot_options* opt,
                               double* const* rho, double* const* phi, double* const* s, double* cost,
                               ot_stats* stats, int32_t* status, int32_t n_streams);

/* One Newton direction at (phi, rho, s) for barrier parameter mu: the solution
 * of the Jacobian system (Eq. newton-linsys) obtained from the projected
 * saddle system (Eq. newton-linsys-shift-reduced-projected) by FGMRES + BB,
 * with the per-slice constants of the splitting (Eq. correction-discrete) and
 * sum(M dphi) = 0.  Outputs dphi ((K+1) x N), drho, ds (K x N'). */
ot_status ot_newton_solve(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho,
                          const double* s, const double* rho_in, const double* rho_f, const ot_options* opt,
                          double* dphi, double* drho, double* ds, ot_stats* stats, void* cuda_stream);

/* Gradient of the discrete cost C with respect to rho_in and rho_f at a
 * converged point (phi, rho, s) of the barrier problem with parameter mu:
 * one adjoint solve with the transposed Jacobian, which after eliminating ds
 * is the same symmetric saddle operator, preconditioned by BB.  Outputs
 * grad_in, grad_f (N' each).  Only mass-preserving perturbations of the
 * densities are admissible (their masses must stay equal), so each gradient
 * is defined up to a multiple of the cell areas |c'|; it is returned in the
 * area gauge, with that component removed (|c'| . grad = 0). */
ot_status ot_cost_grad(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho,
                       const double* s, const double* rho_in, const double* rho_f, const ot_options* opt,
                       double* grad_in, double* grad_f, void* cuda_stream);

/* Autotuner for the multigrid settings of the BB preconditioner (the paper
 * fixes them once for its AGMG solves; choosing them by timed trials has no
 * counterpart there).  For each of n_cand candidates (smooth_sweeps,
 * coarse_sweeps, lap_cycles), given as a host array cand of 3 n_cand int32
 * (NULL: a built-in grid of 12, n_cand ignored), one Newton direction is
 * computed at the state (phi, rho, s) with barrier mu, as by ot_newton_solve
 * with *opt and that candidate's settings, after one untimed solve with *opt
 * itself.  Each trial's wall time (host clock around the solve, which returns
 * after a stream synchronisation) goes to seconds[i] (host, nullable; the
 * built-in grid needs 12 entries), or -1 where the solve failed.  The
 * fastest successful candidate's three settings are written into *opt, the
 * rest of *opt is unchanged.  The state comes in opt->memspace as in
 * ot_newton_solve; the directions are discarded.  Choose the state from the
 * stage whose solves dominate (late, small mu, for a full solve).  Returns the
 * first trial's error if every candidate failed. */
ot_status ot_tune_newton(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho, const double* s,
                         const double* rho_in, const double* rho_f, ot_options* opt, int32_t n_cand,
                         const int32_t* cand, double* seconds, void* cuda_stream);

/* Message for the last failing call on this thread ("" if none). */
const char* ot_last_error(void);

/* ------------------------------------------------------------------------
 * Operator-level entry points (device pointers, float64, the same layouts).
 * They expose single steps of the path so that each can be checked on its
 * own; the solver calls the same kernels.
 * ---------------------------------------------------------------------- */

/* Residual of Eq. (l2-discrete): F_phi ((K+1) x N), F_rho (K x N'),
 * F_s - mu (K x N'); norms (host, 4 doubles, nullable) receives
 * ||F_phi||, ||F_rho||, ||F_s - mu||, ||F||. */
ot_status ot_residual(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho, const double* s,
                      const double* rho_in, const double* rho_f, double* F_phi, double* F_rho, double* F_s,
                      double* norms, void* cuda_stream);

/* y = [A, B^T P^T; P B, -P C P^T] x, the projected saddle operator of
 * Eq. (newton-linsys-shift-reduced-projected); x, y have (K+1) N + K N' entries. */
ot_status ot_kkt_apply(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* s,
                       const double* rho_in, const double* rho_f, const double* x, double* y, void* cuda_stream);

/* The projected saddle operator of ot_kkt_apply, for callers that cannot
 * allocate device memory: a process whose device memory is already reserved
 * by another allocator (a framework's caching pool, a fixed serving budget)
 * where one more cudaMalloc fails or fragments the pool, or a latency-bound
 * loop that cannot afford the device-wide synchronisation cudaMalloc and
 * cudaFree imply.  The paper has no counterpart: this is an interface choice.
 * It allocates nothing and needs no mesh object: n is the number of squares
 * per side (the mesh of ot_mesh_create), K the number of density slices.  Its
 * only scratch (the K slice means of x_rho) is a file-scope device array of
 * 4096 doubles (32 KB) that every GPU loading the library keeps until the
 * process exits; K > 4096 returns OT_ERR_INVALID_ARG.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * device current, so make the first call on each device before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (on
 * different streams at the same time) race on it; each call overwrites all K
 * entries it reads, so nothing has to be cleared.  Device pointers; returns
 * after y is written. */
ot_status ot_kkt_apply_noalloc(int32_t n, int32_t K, const double* phi, const double* rho, const double* s,
                               const double* rho_in, const double* rho_f, const double* x, double* y,
                               void* cuda_stream);

/* out = (Diag(s) A~ - Diag(rho) B M^{-1} B~) z, the operator of Eq. (pseudoschur-bis); z, out K x N'. */
ot_status ot_schur_apply(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* s,
                         const double* z, double* out, void* cuda_stream);

/* One application of the BB preconditioner (Sec. 4.3): given (c; d) returns
 * (x; y) with y = M'^{-1} A~ z, (Diag(s) A~ - Diag(rho) B M^{-1} B~) z ~= -Diag(rho) d
 * and A^k x^k ~= (c - B^T P^T y)^k for every slice (inexact inner solves). */
ot_status ot_bb_apply(ot_mesh* mesh, int32_t K, const ot_options* opt, const double* phi, const double* rho,
                      const double* s, const double* rho_in, const double* rho_f, const double* v, double* out,
                      void* cuda_stream);

/* One application of the SIMPLE preconditioner (Sec. 4.2) to the projected
 * system with A^ = Diag(A): given v = (c; d) (device FP64, (K+1) N + K N'),
 * returns out = (x; y) with
 *   x1 = A^-1 c,  y ~= S^-1 (d - P B x1),  x = x1 - A^-1 B^T P^T y,
 *   S^ = -(P C P^T + P B A^-1 B^T P^T),
 * y in the range of P^T (zero slice means), the Schur solve by GMRES to
 * opt->eps_schur relative residual within opt->schur_max_iter iterations.  At
 * the state (phi, rho, s) (device FP64).  The library allocates and keeps the
 * SIMPLE workspace on first use with this mesh and K. */
ot_status ot_simple_apply(ot_mesh* mesh, int32_t K, const ot_options* opt, const double* phi, const double* rho,
                          const double* s, const double* rho_in, const double* rho_f, const double* v, double* out,
                          void* cuda_stream);

/* Discrete cost C and dual value D (host outputs, nullable). */
ot_status ot_cost_dual(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* rho_in,
                       const double* rho_f, double* cost, double* dual, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Kernel timing (measurement only, off by default).  When on, every launch of
 * an instrumented kernel group is bracketed by CUDA events on its stream and
 * the elapsed device time, the launch count and the algorithmic bytes of the
 * launch (the traffic the operation needs, not what the kernel does) are
 * accumulated; they are collected at the library's stream synchronisations.
 * ---------------------------------------------------------------------- */

/* Turn the accounting on for the groups whose bit is set in group_mask (bit i =
 * group i; -1 = all, 0 = off), timing one launch in `sample_every` (>= 1) of
 * each group; every call resets the counters. */
void ot_kernel_timing_enable(int32_t group_mask, int32_t sample_every);

/* Number of instrumented kernel groups. */
int32_t ot_kernel_timing_count(void);

/* Kernel launches made by this library since it was loaded (all kernels, counted on the host). */
int64_t ot_kernel_launches(void);

/* Counters of group i: name (static string), total milliseconds, launches, bytes. */
ot_status ot_kernel_timing_read(int32_t i, const char** name, double* ms, int64_t* launches, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* OT_H */
