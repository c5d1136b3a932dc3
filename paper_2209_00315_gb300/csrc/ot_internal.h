// ot_internal.h -- kernel launchers and device-memory helpers.
//
// The host orchestration (solver.cpp, capi.cpp) is plain C++: it sees device
// memory only through the dev:: helpers and kernels only through the
// launchers below, all of which enqueue work on the given stream.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <stdexcept>
#include <string>

#include "stencil.cuh"

namespace ot {

typedef void* Stream;  // cudaStream_t

// Error carrying an ot_status code.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

namespace dev {
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
  COUNT
};
extern bool enabled;        // any group on
extern unsigned mask;       // bit i: group i on
extern std::atomic<long long> n_launch;  // kernel launches since load (every launch, timing on or off)
// Timing is per process and single-stream: threads that drive concurrent
// solves (ot_ipm_solve_batched) set `suspended` and are never timed.
extern thread_local bool suspended;
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
};

template <typename T>
void k_mg_lap_coef0(const Dims& d, const double* rho, const double* r0, const double* r1, T* alpha, Stream st);
template <typename T>
void k_mg_schur_coef0(const Dims& d, const double* phi, const double* rho, const double* s, T* alpha, T* tau,
                      Stream st);
template <typename T>
void k_mg_restrict_coef(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st);
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
// Shared memory the fused cycle over these levels needs; it must stay <= kFusedSmemLimit.
template <typename T>
size_t k_mg_fused_smem(int S, const LevelView<T>* levels, int nlev);
constexpr size_t kFusedSmemLimit = 200 * 1024;
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
