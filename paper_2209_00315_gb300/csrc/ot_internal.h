// ot_internal.h -- kernel launchers and device-memory helpers.
//
// The host orchestration (solver.cpp, capi.cpp) is plain C++: it sees device
// memory only through the dev:: helpers and kernels only through the
// launchers below, all of which enqueue work on the given stream.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "stencil.cuh"

namespace ot {

typedef void* Stream;  // cudaStream_t

// Error carrying an ot_status code.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

namespace dev {
// Programmatic dependent launch for this thread's launches (set per solve from
// ot_options.pdl): each kernel may be scheduled while its predecessor's last
// blocks finish; every kernel begins by waiting for its predecessor's results
// (griddepcontrol.wait), so the order of work and its results are unchanged.
extern thread_local bool pdl;
struct PdlScope {
  bool saved;
  explicit PdlScope(bool on) : saved(pdl) { pdl = on; }
  ~PdlScope() { pdl = saved; }
};
void* alloc(size_t bytes);                       // throws Error(OT_ERR_OOM)
// This thread's later alloc/release become stream-ordered on s (null: plain).
void set_alloc_stream(Stream s);
// Bytes the outer Krylov basis of one solve may take on this thread (64 GiB
// unless set; concurrent solves share a budget).
size_t krylov_budget();
void set_krylov_budget(size_t bytes);
void release(void* p);
void* host_alloc(size_t bytes);                  // pinned
void host_release(void* p);
void copy_h2d(void* dst, const void* src, size_t bytes, Stream s);
void copy_d2h(void* dst, const void* src, size_t bytes, Stream s);
void copy_d2d(void* dst, const void* src, size_t bytes, Stream s);
void zero(void* dst, size_t bytes, Stream s);
void sync(Stream s);
void check(const char* where);                   // throws Error(OT_ERR_CUDA) on a pending error
bool is_device_pointer(const void* p);
double now();                                    // seconds, host clock
int current_device();
void set_device(int device);
Stream stream_create();                          // non-blocking stream
void stream_destroy(Stream s);                   // after synchronising it
void sync_quiet(Stream s);                       // synchronise, ignoring errors
}  // namespace dev

// ------------------------------------------------------------------ device-controlled Krylov loops
// State of one (F)GMRES solver kept in device memory, so that an Arnoldi step,
// its convergence test and the decision to run another step need no host
// round trip (and can run inside a captured CUDA graph).
namespace kry {
enum Status { RUNNING = 0, CONVERGED = 1, BREAKDOWN = 2, NONFINITE = 3, LIMIT = 4 };
struct Ctl {
  int j;           // Arnoldi steps done in the current cycle (= index of the next column)
  int m;           // cycle length
  int status;      // Status
  int k;           // columns of the last least-squares solve
  int base;        // steps of the earlier cycles of the current linear solve
  int cap;         // steps allowed per linear solve
  long long total; // steps since the workspace was made (statistics)
  double beta;     // residual norm at the start of the cycle
  double tol;      // absolute stopping tolerance of the linear solve
  double res;      // residual estimate |g_{j}|
  double pad[3];
};
}  // namespace kry
// Condition of a graph's WHILE node (a cudaGraphConditionalHandle); `on` is
// false when the loop runs eagerly, without a graph.
struct CondHandle {
  unsigned long long h = 0;
  bool on = false;
};

namespace dev {
// A loop whose trip count the device decides.  prologue(s, h) enqueues the
// work before the loop and must set ctl->status (and, when h.on, the loop
// condition h); body(s, h, j) enqueues one iteration whose last kernel sets
// both.  When stream st is being captured into a CUDA graph, the loop becomes
// a WHILE conditional node of that graph (the body is captured once into the
// node's body graph, on a helper stream of this thread, with j = -1);
// otherwise the body is enqueued eagerly while ctl->status reads RUNNING (one
// device-to-host read per iteration; j = ctl->j as read).  Returns the kernel
// launches of one body iteration.
long long device_while(Stream st, const kry::Ctl* ctl, const std::function<void(Stream, CondHandle)>& prologue,
                       const std::function<void(Stream, CondHandle, int)>& body);
bool capturing(Stream st);
// Read the control block (device-to-host copy and stream synchronisation).
void read_ctl(const kry::Ctl* ctl, kry::Ctl* out, Stream st);

// One instantiated CUDA graph made by capturing `enqueue` on a private stream.
struct Graph {
  void* exec = nullptr;      // cudaGraphExec_t
  void* graph = nullptr;     // cudaGraph_t
  long long static_launches = 0;                      // kernel launches outside loops
  // per loop, in capture order: its control block and the launches of one
  // iteration outside nested loops
  std::vector<std::pair<const kry::Ctl*, long long>> loops;
  void capture(const std::function<void(Stream)>& enqueue);
  void launch(Stream st);
  // kernel launches of one run whose loops made iterations[i] iterations
  long long executed(const std::vector<long long>& iterations) const;
  void release();
  bool ready() const { return exec != nullptr; }
  ~Graph() { release(); }
};
}  // namespace dev

// ------------------------------------------------------------------ kernel timing
// Opt-in device-time accounting: when enabled, instrumented launchers bracket
// their launch with CUDA events on the launching stream; dev::sync() harvests
// the finished pairs.  `bytes` is the algorithmic traffic of the launch.
namespace prof {
enum Id {
  KKT = 0,       // projected KKT operator (4 kernels)
  MDOT,          // Gram-Schmidt dot products
  MUPDATE,       // Gram-Schmidt update (+ fused dots / norm)
  MCOMBINE,      // x += Z y
  LAP_SMOOTH,    // red-black point Gauss-Seidel, slice Laplacians
  SCH_SMOOTH,    // red-black line Gauss-Seidel, Schur space-time operator
  MG_TRANSFER,   // residual, restriction, prolongation
  SCHUR,         // Schur operator (2 kernels)
  RESIDUAL,      // residual F
  BT,            // B^T P^T y
  LAP_LOWER,     // fused small levels of a slice-Laplacian V-cycle (one launch)
  SCH_LOWER,     // fused small levels of a space-time Schur V-cycle (one launch)
  SIMPLE_LINE,   // time-line solves preconditioning SIMPLE's Schur complement
  COUNT
};
extern bool enabled;        // any group on
extern unsigned mask;       // bit i: group i on
extern std::atomic<long long> n_launch;  // kernel launches since load (every launch, timing on or off)
// Timing is per process and single-stream: threads that drive concurrent
// solves (ot_ipm_solve_batched) set `suspended` and are never timed.
extern thread_local bool suspended;
// Set while this thread captures a CUDA graph: no event pairs are recorded
// (a captured launch has no per-launch events).
extern thread_local bool capturing;
extern thread_local long long t_captured;  // launches this thread has captured into graphs
extern int stride;          // time one launch in `stride` of each enabled group
void begin(int id, Stream s);
void end(int id, Stream s, double bytes);
void harvest();
void reset();
const char* name(int id);
void read(int id, double* ms, long long* launches, double* bytes);
}  // namespace prof

// ------------------------------------------------------------------ reductions / BLAS-1
// sums[k] = scale * sum_i x[k*n + i], k < S.
void k_slice_sums(const double* x, int S, i64 n, double scale, double* sums, Stream s);
// x[k*n + i] -= sums[k] * scale (remove slice means when scale = 1/n).
void k_slice_shift(double* x, int S, i64 n, const double* sums, double scale, Stream s);
// out[v] = <V_v, w>, v < nv; V_v = V + v*ld.  partial: scratch of k_reduce_scratch(nv) doubles.
void k_mdot(const double* V, i64 ld, int nv, const double* w, i64 n, double* out, double* partial, Stream s);
// w -= sum_v h[v] V_v; then out[v] = <V_v, w_new> (if out) and out[nv] = <w_new, w_new> (if norm).
void k_mupdate(const double* V, i64 ld, int nv, const double* h, double* w, i64 n, double* out, bool dots,
               bool norm, double* partial, Stream s);
// x += sum_v y[v] Z_v
void k_mcombine(const double* Z, i64 ld, int nv, const double* y, double* x, i64 n, Stream s);
// out[0] = <x, y>
void k_dot(const double* x, const double* y, i64 n, double* out, double* partial, Stream s);
// y = a x + b y
void k_axpby(double a, const double* x, double b, double* y, i64 n, Stream s);
// y = x / sqrt(nrm2[0])  (nrm2 in device memory)
void k_scale_by_inv_norm(const double* x, const double* nrm2, double* y, i64 n, Stream s);
// y = x * a
void k_scale(const double* x, double a, double* y, i64 n, Stream s);
void k_fill(double* x, double v, i64 n, Stream s);
size_t k_reduce_scratch(int nv);  // doubles needed by `partial`

// ------------------------------------------------------------------ device-controlled Arnoldi steps
// The vector counts of these kernels are read from the control block (nv =
// ctl->j + add) and their grids depend only on the basis size mmax, so one
// capture serves every step.  Coefficients and norms are double; T is the
// basis precision (double, or float for the inner Schur solve).
size_t kry_partial_doubles(int mmax);  // scratch doubles of kry_dot / kry_update (incl. an arrival counter)
size_t kry_counter_offset(int mmax);   // first double of the arrival counter inside that scratch
// The Givens step of an Arnoldi iteration (column j of the Hessenberg matrix
// from the two Gram-Schmidt passes, hc1 nullable; the earlier rotations and the
// new one; residual estimate, status, j += 1, loop condition h), taken by the
// last block of the update that produces |w|^2.
struct KryGivens {
  kry::Ctl* ctl;
  const double* hc1;
  const double* hc2;
  double* H;
  int ldh;
  double* cs;
  double* sn;
  double* g;
  unsigned long long h;
  int on;
};
// out[v] = <V_v, w>, v < nv.
// nv_hint: nv when the host knows it (eager loops; kernel-timing bytes only), else -1.
template <typename T>
void kry_dot(const T* V, i64 ld, const kry::Ctl* ctl, int add, int mmax, const T* w, i64 n, double* out,
             double* partial, int nv_hint, Stream s);
// w -= sum_{v < nv} h[v] V_v; w32 (nullable) receives the new w in float;
// norm_out (nullable): norm_out[nv] = |new w|^2, followed by the Givens step gv
// (nullable) in the same launch.
template <typename T>
void kry_update(const T* V, i64 ld, const kry::Ctl* ctl, int add, int mmax, const double* h, T* w, i64 n,
                float* w32, double* norm_out, double* partial, int nv_hint, Stream s, const KryGivens* gv = nullptr);
// The same update of an FP64 w from an FP32 basis (the FP32 copy of V), the
// combination formed in FP32: for the second Gram-Schmidt pass, whose
// coefficients are ~1e-7 of |w|.
void kry_update_shadow(const float* V32, i64 ld, const kry::Ctl* ctl, int add, int mmax, const double* h, double* w,
                       i64 n, double* norm_out, double* partial, int nv_hint, Stream s,
                       const KryGivens* gv = nullptr);
// With j = ctl->j + add: V_{j+1} = w / sqrt(nrm2[j+1]); V32 (nullable) and copy
// (nullable) receive it too; Z_j = zsrc when zsrc is given.
template <typename T>
void kry_next_basis(const T* w, const double* nrm2, const kry::Ctl* ctl, int add, T* V, i64 ld, float* V32, T* copy,
                    const T* zsrc, T* Z, i64 n, Stream s);
// V0 = r / sqrt(nrm2[0]); V32_0 (nullable) and copy (nullable) receive it too.
template <typename T>
void kry_start_basis(const T* r, const double* nrm2, T* V0, float* V32_0, T* copy, i64 n, Stream s);
// Once per linear solve: base = 0, cap, tol = tol_rel * sqrt(sum_{i < nref} ref[i]) (nref > 0).
void kry_solve_init(kry::Ctl* ctl, const double* ref, int nref, double tol_rel, int cap, Stream s);
// Start of a cycle: beta = sqrt(nrm2[0]), g[0] = beta, j = 0; with tol_rel > 0 the
// tolerance becomes tol_rel * beta; status RUNNING unless beta is already small
// enough (or not finite); the loop condition h (if any) follows the status.
void kry_start(kry::Ctl* ctl, const double* nrm2, int m, double tol_rel, double* g, CondHandle h, Stream s);
// y = R^{-1} g over the ctl->j columns (ctl->k = j, ctl->base += j).
void kry_backsolve(kry::Ctl* ctl, const double* H, int ldh, const double* g, double* y, Stream s);
// x += sum_{v < ctl->k} y[v] Z_v
template <typename T>
void kry_combine(const T* Z, i64 ld, const kry::Ctl* ctl, int mmax, const double* y, T* x, i64 n, int nv_hint,
                 Stream s);

// FP32 overloads (mixed precision: the preconditioner's inner Krylov solve).
// Per-thread accumulation is in float; cross-thread reductions and the
// scalars (h, y, out, partial) are double.
void k_slice_sums(const float* x, int S, i64 n, double scale, float* sums, Stream s);
void k_slice_shift(float* x, int S, i64 n, const float* sums, double scale, Stream s);
void k_mdot(const float* V, i64 ld, int nv, const float* w, i64 n, double* out, double* partial, Stream s);
void k_mupdate(const float* V, i64 ld, int nv, const double* h, float* w, i64 n, double* out, bool dots,
               bool norm, double* partial, Stream s);
void k_mcombine(const float* Z, i64 ld, int nv, const double* y, float* x, i64 n, Stream s);
void k_dot(const float* x, const float* y, i64 n, double* out, double* partial, Stream s);
void k_scale_by_inv_norm(const float* x, const double* nrm2, float* y, i64 n, Stream s);
void k_scale(const float* x, double a, float* y, i64 n, Stream s);

// ------------------------------------------------------------------ operators (FP64)
void k_residual(const Dims& d, double mu, const double* phi, const double* rho, const double* s,
                const double* r0, const double* r1, double* Fphi, double* Frho, double* Fs, Stream st);
// Edge coefficients of the KKT operator at (phi, rho, s): kc holds
// kkt_coef_count(d) doubles (layout in stencil.cuh).
void k_kkt_coef(const Dims& d, const double* phi, const double* rho, const double* s, const double* r0,
                const double* r1, double* kc, Stream st);
// xmean[K] = slice means of x_rho; y = projected KKT operator (coefficients kc) applied to x.
// wsum (nullable, K): slice sums of B x_phi - C P^T x_rho before the projection.
void k_kkt_apply(const Dims& d, const double* kc, const double* x, double* y, double* xmean, double* wsum,
                 Stream st);
// The same operator with its slice-mean scratch in a file-scope device array
// (no allocation); K <= kStaticKktMaxK.  The first call on a device resolves
// the array's address (cudaGetSymbolAddress) with that device current.
constexpr int kStaticKktMaxK = 4096;
constexpr int kStaticKktMaxDevices = 64;
void k_kkt_apply_static(const Dims& d, const double* phi, const double* rho, const double* s, const double* r0,
                        const double* r1, const double* x, double* y, Stream st);
// y_phi = B^T P^T y_rho (phi rows only, no A term) from the KKT coefficients kc; yr_mean: scratch K.
void k_bt_apply(const Dims& d, const double* kc, const double* yr, double* out_phi, double* yr_mean, Stream st);
// Schur operator of Eq. (pseudoschur-bis); u: scratch (K+1) N.
void k_schur_apply(const Dims& d, const double* phi, const double* rho, const double* s, const double* z,
                   double* out, double* u, Stream st);
// y = M'^{-1} A~ z
void k_atilde_minv(const Dims& d, const double* rho, const double* z, double* y, Stream st);
// cost: out[0] = C, dual: out[1] = D.
void k_cost_dual(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                 double* out, double* partial, Stream st);
// Newton RHS from the residual: f = -F_phi, h = -(F_s - mu), gt = P(-F_rho - |c'| h/rho) written to
// rhs = (f; gt); gsum[K] = slice sums of g~ before the projection.
void k_newton_rhs(const Dims& d, const double* Fphi, const double* Frho, const double* Fs, const double* rho,
                  double* rhs, double* hvec, double* gsum, Stream st);
// ds = (h - s drho)/rho ; returns via out[0] the largest step in (0, inf] keeping rho, s > 0 scaled by tau.
void k_step_length(const Dims& d, const double* rho, const double* s, const double* drho, const double* hvec,
                   double* ds, double tau, double* out, double* partial, Stream st);
// phi += a dphi, rho += a drho, s += a ds with a = alpha_dev[0] (device) or a_host if alpha_dev is null.
void k_update(const Dims& d, const double* alpha_dev, double a_host, const double* dphi, const double* drho,
              const double* ds, double* phi, double* rho, double* s, Stream st);
// Per-slice constants of the splitting (reading R10): cshift[0] = 0,
// cshift[j+1] = cshift[j] + dt (gsum[j] - wsum[j]) / area_total, j < K.
void k_shift_constants(const Dims& d, const double* gsum, const double* wsum, double area_total, double* cshift,
                       Stream st);
// rho^k *= target / mass[k]
void k_rescale(const Dims& d, double* rho, const double* mass, double target, Stream st);
// Initial point (reading R8).
void k_init_point(const Dims& d, double mu0, const double* r0, const double* r1, double* phi, double* rho,
                  double* s, Stream st);
// out = scale * a .* b
void k_mul(const double* a, const double* b, double scale, double* out, i64 n, Stream st);
// Adjoint right-hand side dC/d(phi, rho) written as (c_phi; P c_rho); gsum[K] = slice sums of c_rho.
void k_adjoint_rhs(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                   double* rhs, double* gsum, Stream st);
// grad_in, grad_f (N' each) from the adjoint potential lam ((K+1) x N).
void k_adjoint_grad(const Dims& d, const double* phi, const double* lam, double* gin, double* gf, Stream st);
// 3D Cartesian variant (k_cube.cu): n^3 cubes, J = I; operator level only.
struct CubeDims {
  int n, K;
  i64 N;       // cells (= n^3, density and potential alike)
  double h, V, T, dt;  // side, volume, face transmissibility |e|/|w| = h, 1/(K+1)
};
CubeDims make_cube_dims(int n, int K);
void k_cube_residual(const CubeDims& d, double mu, const double* phi, const double* rho, const double* s,
                     const double* r0, const double* r1, double* Fphi, double* Frho, double* Fs, Stream st);
// y = projected KKT operator applied to x; scratch: 2 K doubles.
void k_cube_kkt_apply(const CubeDims& d, const double* phi, const double* rho, const double* s, const double* r0,
                      const double* r1, const double* x, double* y, double* scratch, Stream st);
// out[0] = C, out[1] = D; scratch: 2 N doubles.
void k_cube_cost_dual(const CubeDims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                      double* out, double* scratch, Stream st);
// SIMPLE preconditioner pieces (k_simple.cu).  Ad ((K+1) N) = diagonal of the
// potential block A from the KKT coefficients kc.
void k_simple_diag(const Dims& d, const double* kc, double* Ad, Stream st);
// Factors (inv, e: K x N' each) of the time-line tridiagonal systems that
// precondition SIMPLE's Schur complement, from kc and Ad.
void k_simple_line_factor(const Dims& d, const double* kc, const double* Ad, double* inv, double* e, Stream st);
// z = L^-1 (r - shift), L the time-line tridiagonal systems per coarse cell;
// shift (nullable, K) is subtracted slice by slice; r and z (K x N') may not alias.
void k_simple_line_solve(const Dims& d, const double* inv, const double* e, const double* r, const double* shift,
                         double* z, Stream st);
// G = Y^T L^-1 Y (K x K, Y the slice indicators), Cholesky-factored in place
// (lower, column-major); scratch: K x N'; *status set to 1 if a pivot is not positive.
constexpr int kSimpleMaxK = 1024;
void k_simple_gram(const Dims& d, const double* inv, const double* e, double* scratch, double* G, int* status,
                   Stream st);
// lam = G^-1 t from the factor of k_simple_gram (K <= kSimpleMaxK).
void k_simple_gram_solve(int K, const double* L, const double* t, double* lam, Stream st);
// out = beta * out + alpha * num / den (element-wise; beta = 0 ignores out's old values)
void k_quot(const double* num, const double* den, double alpha, double* out, double beta, i64 n, Stream st);
// FP32 versions of the Schur-side operators (mixed precision), same layouts.
void k_bt_apply(const Dims& d, const float* phi, const float* yr, float* out_phi, float* yr_mean, Stream st);
void k_schur_apply(const Dims& d, const float* phi, const float* rho, const float* s, const float* z, float* out,
                   float* u, Stream st);
void k_atilde_minv(const Dims& d, const float* rho, const float* z, float* y, Stream st);
// dst = scale * src, converting precision
void k_convert(const double* src, float* dst, i64 n, double scale, Stream st);
void k_convert(const float* src, double* dst, i64 n, double scale, Stream st);
// out = (float)(scale * a .* b)
void k_mul(const float* a, const double* b, double scale, float* out, i64 n, Stream st);
// y = c - y
void k_rsub(const double* c, float* y, i64 n, Stream st);
// max |x| and non-finite flag: out[0] = max|x|, out[1] = 1 if any non-finite
void k_absmax(const double* x, i64 n, double* out, double* partial, Stream st);
// min(x) -> out[0]
void k_min(const double* x, i64 n, double* out, double* partial, Stream st);

// ------------------------------------------------------------------ multigrid (T = float or double)
// Level arrays are slice-major with slice stride ld: cell c of slice k is
// element k*ld + c (alpha: (slot*S + k)*ld + c).  Device-memory levels have
// ld == nc; shared-memory copies pad ld to an odd stride so that the 32 lanes
// of a time line hit 32 different banks.
template <typename T>
struct LevelView {
  int m;        // grid side
  i64 nc;       // cells per slice
  i64 ld;       // slice stride, >= nc
  T* alpha;     // [3][S][ld]
  T* tau;       // [S][ld] or nullptr
  T* x;
  T* b;
  T* r;
  // Thomas factors of the time lines, [2][S][ld] (1/pivot, then the modified
  // upper coefficient), on the space-time levels swept by tiles (device memory,
  // refreshed with the coefficients) and on the shared-memory copies of the
  // fused levels (factored at the start of each fused cycle); nullptr elsewhere.
  // The line systems change once per Newton step; every sweep only substitutes.
  T* fac = nullptr;
  // Shared-memory copies of the fused levels only: per cell its three
  // neighbours (-1 on the boundary) [3][nc], its parent on the next coarser
  // level [nc] (-1 on the coarsest), its four children on the next finer level
  // [4][nc] (level 0: unused); built once per fused launch, so that sweeps and
  // transfers index with 32-bit loads instead of decoding cell numbers.
  int* nbt = nullptr;
  int* par = nullptr;
  int* chd = nullptr;
};

template <typename T>
void k_mg_lap_coef0(const Dims& d, const double* rho, const double* r0, const double* r1, T* alpha, Stream st);
template <typename T>
void k_mg_schur_coef0(const Dims& d, const double* phi, const double* rho, const double* s, T* alpha, T* tau,
                      Stream st);
template <typename T>
void k_mg_restrict_coef(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st);
// Thomas factors of every time line of a space-time level (L.fac in device
// memory; nothing if the level has none): once per Newton step, after the coefficients.
template <typename T>
void k_mg_line_factor(int S, const LevelView<T>& L, Stream st);
template <typename T>
void k_mg_smooth(int S, const LevelView<T>& L, int color, T* line_c, T* line_r, Stream st);
// A sweep of one colour in a mode: 0 plain; 1 the first sweep from x = 0
// (neighbour values taken as zero, x need not be initialised); 2 the first
// sweep after a coarse correction (neighbour values x + J x_coarse; the
// correction itself is never stored, because the next sweep of the other
// colour overwrites those cells without reading them).
template <typename T>
void k_mg_smooth_mode(int S, const LevelView<T>& L, const LevelView<T>* coarse, int color, int mode, T* line_c,
                      T* line_r, Stream st);
template <typename T>
void k_mg_residual(int S, const LevelView<T>& L, Stream st);
// b_coarse = J^T (b - M x) in one pass (no fine residual stored)
template <typename T>
void k_mg_restrict_residual(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st);
template <typename T>
void k_mg_restrict(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st);
template <typename T>
void k_mg_prolong(int S, const LevelView<T>& coarse, const LevelView<T>& fine, Stream st);
template <typename T>
void k_mg_coarse_solve(int S, const LevelView<T>& L, int sweeps, T* line_c, T* line_r, T* agg, Stream st);
// The V-cycle from levels[0] to levels[nlev-1] (the coarsest) in one launch: x
// of every level zeroed, nu pre/post sweeps, nuc sweeps (and, for the
// space-time hierarchy, the aggregate correction) on the coarsest level.
template <typename T>
void k_mg_lower_cycle(int S, const LevelView<T>* levels, int nlev, int nu, int nuc, T* line_c, T* line_r, T* agg,
                      Stream st);
// Grant the fused cycle's kernel the shared memory these levels need (once,
// before any stream capture: a capture cannot change kernel attributes).
template <typename T>
void k_mg_prepare_lower_cycle(int S, const LevelView<T>* levels, int nlev);
// Shared memory the fused cycle over these levels needs; it must stay <= kFusedSmemLimit.
template <typename T>
size_t k_mg_fused_smem(int S, const LevelView<T>* levels, int nlev);
constexpr size_t kFusedSmemLimit = 220 * 1024;
// b = (T)(scale * src); x = 0
template <typename T>
void k_mg_load(const double* src, double scale, T* b, T* x, i64 n, Stream st);
// dst = (double) x
template <typename T>
void k_mg_store(const T* x, double* dst, i64 n, Stream st);
// y += a x
template <typename T>
void k_mg_axpy(const T* x, T a, T* y, i64 n, Stream st);

}  // namespace ot
