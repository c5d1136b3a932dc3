// solver.h -- workspace and host orchestration of the IPM / FGMRES / BB path.
#pragma once
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/ot.h"
#include "ot_internal.h"

namespace ot {

// Multigrid hierarchy on nested grids of sides m0, m0/2, ... (down to an odd side).
template <typename T>
struct Hierarchy {
  int S = 0;               // slices
  bool time_coupled = false;
  std::vector<LevelView<T>> lv;
  T* line_c = nullptr;     // Thomas scratch, S x nc(level 0)
  T* line_r = nullptr;
  T* agg = nullptr;        // 4 S
  T* acc = nullptr;        // level-0 accumulator for repeated cycles
  T* bsave = nullptr;      // level-0 right-hand side for repeated cycles
  size_t fuse_from = 0;    // first level handled by the fused lower-cycle kernel (lv.size(): none)
  void build(int m0, int S, bool time_coupled);
  void release();
  bool built() const { return !lv.empty(); }
};

// Krylov basis storage for one (F)GMRES solver; the basis in T, the
// Hessenberg columns and coefficients in double.
template <typename T>
struct KrylovT {
  int mmax = 0;
  i64 n = 0;
  T* V = nullptr;          // (mmax+1) x n
  T* Z = nullptr;          // mmax x n
  T* w = nullptr;          // n
  T* in = nullptr;         // n: the newest basis vector, the preconditioner's input
  T* zout = nullptr;       // n: the preconditioner's output, before it is stored in Z
  double* hc1 = nullptr;   // mmax+2
  double* hc2 = nullptr;   // mmax+2
  double* y = nullptr;     // mmax+2
  // FP32 shadow of V and w (shadow = true): the Gram-Schmidt dot products are
  // taken from them in FP32 (the first pass always, the second when the solve's
  // target allows); the coefficients are applied to the FP64 basis.
  float* V32 = nullptr;    // (mmax+1) x n
  float* w32 = nullptr;    // n
  // device-side iteration state (k_krylov.cu)
  kry::Ctl* ctl = nullptr;
  double* H = nullptr;     // (mmax+1) x mmax, column-major, leading dimension mmax+1
  double* cs = nullptr;    // mmax+1
  double* sn = nullptr;    // mmax+1
  double* g = nullptr;     // mmax+2
  double* part = nullptr;  // kry_partial_doubles(mmax)
  double* scal = nullptr;  // 8: [0] squared norm of the cycle's start vector
  void build(int m, i64 n, bool shadow = false);
  void release();
  int ldh() const { return mmax + 1; }
};
typedef KrylovT<double> Krylov;

// The BB preconditioner's vectors in the precision T of its Schur solve.  For
// T = double the state pointers alias the FP64 state; for T = float they are
// copies refreshed with the coefficients once per Newton step.
template <typename T>
struct BBVectors {
  const T *phi = nullptr, *rho = nullptr, *s = nullptr;
  T* u = nullptr;       // Schur scratch, (K+1) N
  T* srhs = nullptr;    // Nr
  T* zeta = nullptr;    // Nr
  T* y = nullptr;       // Nr (T = float only: y before conversion)
  T* bphi = nullptr;    // Np
  T* mean = nullptr;    // K+2
  T* sums = nullptr;    // K+2
  KrylovT<T>* K = nullptr;
};

// Everything one (mesh, K, precision) needs on the device.
struct Workspace {
  Dims d;
  int precision = OT_PREC_FP64;
  i64 Np = 0, Nr = 0, ntot = 0;
  // state
  double *phi = nullptr, *rho = nullptr, *s = nullptr, *r0 = nullptr, *r1 = nullptr;
  // residual and Newton
  double *Fphi = nullptr, *Frho = nullptr, *Fs = nullptr;
  double *rhs = nullptr, *sol = nullptr, *hvec = nullptr, *ds = nullptr, *ytmp = nullptr;
  double *gsum = nullptr, *wsum = nullptr, *cshift = nullptr, *xmean = nullptr, *mass = nullptr;
  double* kcoef = nullptr;    // KKT edge coefficients at the current state (kkt_coef_count doubles)
  double* scal = nullptr;     // 64 device scalars
  double* partial = nullptr;  // reduction scratch
  // BB
  double *u = nullptr, *bphi = nullptr, *srhs = nullptr, *zeta = nullptr;
  Krylov outer, inner;
  KrylovT<float> innerf;
  float* f32 = nullptr;       // one allocation for the FP32 vectors of mixed precision
  float *phif = nullptr, *rhof = nullptr, *sf = nullptr;
  BBVectors<double> bbd;
  BBVectors<float> bbf;
  Hierarchy<float> lapf, schf;
  Hierarchy<double> lapd, schd;
  // SIMPLE (allocated on first use): the diagonal of A, the time-line factors of
  // its Schur complement's preconditioner, and a KKT input vector
  double *sAd = nullptr, *sinv = nullptr, *se = nullptr, *skin = nullptr;
  double *sG = nullptr, *slam = nullptr;  // Cholesky factor of Y^T L^-1 Y (K x K); 2 K scalars
  int* sstat = nullptr;                   // factorisation status (device)
  double mu = 1.0;            // barrier parameter of the Newton system being solved
  double* host = nullptr;     // pinned host scratch: [0, hoff) and [hoff, 2 hoff) Hessenberg columns, then 64 scalars
  int hoff = 0;
  // counters of the current call
  long long outer_iters = 0, inner_iters = 0, capped_solves = 0;
  int cur_restart = 0, cur_inner = 0;
  // captured FGMRES cycles (one graph per configuration of the cycle)
  std::map<std::string, std::unique_ptr<dev::Graph>> graphs;

  Workspace(int n, int K, int precision, const ot_options& opt);
  ~Workspace();
};

constexpr int kMaxRestart = 800;

// FGMRES restart length for these options and ntot unknowns: opt.fgmres_restart
// if > 0; otherwise (automatic) the iteration cap, i.e. no restart as in the
// paper, as far as the Krylov basis (V, Z and V's FP32 shadow) fits the thread's budget
// (dev::krylov_budget), never below 30.
int effective_restart(const ot_options& opt, i64 ntot);

// KKT edge coefficients, level-0 coefficients of both hierarchies and their
// coarsenings (and the FP32 state copies) from the current (phi, rho, s).
void refresh_coefficients(Workspace& W, Stream st);
// One BB preconditioner application (Sec. 4.3): out = P_BB^{-1} v, both of length ntot.
void bb_apply(Workspace& W, const ot_options& opt, const double* v, double* out, Stream st);
// Whether the outer FGMRES at barrier parameter mu uses SIMPLE (opt.precond).
bool use_simple(const ot_options& opt, double mu);
// Allocate SIMPLE's workspace (first use; never inside a graph capture) and
// compute its diagonal and line factors from the current KKT coefficients.
void simple_prepare(Workspace& W, Stream st);
// One SIMPLE application (Sec. 4.2): out = P_SIMPLE^{-1} v, both of length ntot
// (after simple_prepare at the current coefficients).
void simple_apply(Workspace& W, const ot_options& opt, const double* v, double* out, Stream st);
// FGMRES on the projected system; x (ntot) receives the solution; stops at a
// residual estimate <= tol_rel * sqrt(sum_{i < nref} tol_ref[i]) (device
// scalars, squared norms); returns the final residual estimate.
double fgmres(Workspace& W, const ot_options& opt, const double* b, double* x, double tol_rel,
              const double* tol_ref, int nref, Stream st);
// Residual at the state in W for parameter mu; returns ||F|| (norms[0..2]: component norms).
double residual_norm(Workspace& W, double mu, Stream st, double* norms);
// Newton direction at the state in W; requires the residual of that state in W.F*.
// On return: sol = (dphi; drho), ds, and scal[0] = step length (device); returns the step length.
double newton_direction(Workspace& W, const ot_options& opt, double normF, double eps, Stream st);
// Turn the projected solution in W.sol into the full direction (reading R10):
// drho <- P^T drho; dphi <- dphi_hat + per-slice constants from W.gsum; zero mean.
void recover_direction(Workspace& W, Stream st);
// Full interior-point solve from the state in W (initialised by the caller).
int ipm_run(Workspace& W, const ot_options& opt, double mu0, double tol, ot_stats* stats, Stream st);

}  // namespace ot
