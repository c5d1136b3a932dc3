// capi.cpp -- the extern "C" entry points of include/ot.h.
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/ot.h"
#include "solver.h"

using ot::Error;
using ot::i64;
using ot::Stream;
using ot::Workspace;
namespace dev = ot::dev;

struct ot_mesh {
  int kind = OT_MESH_STRUCTURED_SQUARE;
  int n = 0;
  std::map<std::pair<int, int>, std::unique_ptr<Workspace>> ws;
};

// The 3D Cartesian variant runs its operator-level calls on scratch of its own.
static bool is_cube(const ot_mesh* m) { return m && m->kind == OT_MESH_CARTESIAN_CUBE; }
struct CubeScratch {
  double* dev = nullptr;   // max(2 K, 2 N) + 2 doubles
  double* host = nullptr;  // 2 doubles (pinned)
  explicit CubeScratch(size_t n) {
    dev = (double*)dev::alloc(sizeof(double) * n);
    host = (double*)dev::host_alloc(2 * sizeof(double));
  }
  ~CubeScratch() {
    dev::release(dev);
    dev::host_release(host);
  }
};

static thread_local std::string g_err;

static ot_status set_err(int code, const std::string& m) {
  g_err = m;
  return (ot_status)code;
}

#define OT_TRY \
  g_err.clear(); \
  try {
#define OT_CATCH                                                          \
  }                                                                       \
  catch (const Error& e) {                                                \
    return set_err(e.code, e.what());                                     \
  }                                                                       \
  catch (const std::bad_alloc&) {                                         \
    return set_err(OT_ERR_OOM, "host allocation failed");                 \
  }                                                                       \
  catch (const std::exception& e) {                                       \
    return set_err(OT_ERR_CUDA, e.what());                                \
  }

static void require(bool ok, const char* msg) {
  if (!ok) throw Error(OT_ERR_INVALID_ARG, msg);
}

extern "C" {

void ot_default_options(ot_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->memspace = OT_MEM_DEVICE;
  o->precision = OT_PREC_FP64;
  o->mu_factor = 0.2;
  o->tau = 0.99;
  o->newton_tol = 1e-6;
  o->final_newton_tol = 0.0;
  o->eps_out = 1e-5;
  o->final_eps_out = 0.0;
  o->eps_schur = 1e-1;
  o->fgmres_restart = 0;  // automatic: no restart up to the cap, within the Krylov memory budget
  o->fgmres_max_iter = 400;
  o->schur_max_iter = 20;
  o->lap_cycles = 2;     // two V(2,2) cycles: ~5e-2 relative residual, the paper's Laplacian tolerance
  o->smooth_sweeps = 2;
  o->coarse_sweeps = 6;
  o->max_newton = 50;
  o->verbose = 0;
  o->gs_shadow = 1;
  o->graphs = 1;
  o->precond = OT_PRECOND_BB;
  o->simple_mu = 1e-5;
  o->pdl = 1;
}

const char* ot_last_error(void) { return g_err.c_str(); }

}  // extern "C"

static bool supported_side(int n) {
  if (n < 1 || n > 4096) return false;
  while (n % 2 == 0) n /= 2;
  return n <= 11;
}

static ot_options resolve(const ot_options* o) {
  ot_options r;
  if (o)
    r = *o;
  else
    ot_default_options(&r);
  require(r.memspace == OT_MEM_DEVICE || r.memspace == OT_MEM_HOST, "options.memspace");
  require(r.precision == OT_PREC_FP64 || r.precision == OT_PREC_MIXED, "options.precision");
  require(r.mu_factor > 0 && r.mu_factor < 1, "options.mu_factor must be in (0, 1)");
  require(r.tau > 0 && r.tau < 1, "options.tau must be in (0, 1)");
  require(r.newton_tol > 0 && r.eps_out > 0 && r.eps_schur > 0, "tolerances must be positive");
  require(r.fgmres_restart >= 0 && r.fgmres_restart <= ot::kMaxRestart,
          "options.fgmres_restart must be in [0, 800] (0: automatic)");
  require(r.fgmres_max_iter >= 1, "options.fgmres_max_iter");
  require(r.schur_max_iter >= 1 && r.schur_max_iter <= 480, "options.schur_max_iter must be in [1, 480]");
  require(r.lap_cycles >= 1 && r.smooth_sweeps >= 0 && r.coarse_sweeps >= 1, "multigrid cycle counts");
  require(r.max_newton >= 1, "options.max_newton");
  require(r.gs_shadow == 0 || r.gs_shadow == 1, "options.gs_shadow must be 0 or 1");
  require(r.graphs == 0 || r.graphs == 1, "options.graphs must be 0 or 1");
  require(r.precond == OT_PRECOND_BB || r.precond == OT_PRECOND_SIMPLE || r.precond == OT_PRECOND_HYBRID,
          "options.precond must be OT_PRECOND_BB, OT_PRECOND_SIMPLE or OT_PRECOND_HYBRID");
  require(r.simple_mu >= 0 && std::isfinite(r.simple_mu), "options.simple_mu must be finite and >= 0");
  require(r.pdl == 0 || r.pdl == 1, "options.pdl must be 0 or 1");
  return r;
}

static Workspace& workspace(ot_mesh* m, int K, const ot_options& o) {
  require(m != nullptr, "mesh is NULL");
  require(!is_cube(m), "3D Cartesian meshes support only ot_residual, ot_kkt_apply and ot_cost_dual");
  require(K >= 1 && K <= 4096, "K must be in [1, 4096]");
  auto key = std::make_pair(K, o.precision);
  auto it = m->ws.find(key);
  if (it != m->ws.end() &&
      (it->second->cur_restart < ot::effective_restart(o, it->second->ntot) ||
       it->second->cur_inner < o.schur_max_iter))
    m->ws.erase(it), it = m->ws.end();
  if (it == m->ws.end()) {
    auto w = std::unique_ptr<Workspace>(new Workspace(m->n, K, o.precision, o));
    it = m->ws.emplace(key, std::move(w)).first;
  }
  return *it->second;
}

static void copy_in(double* dst, const double* src, i64 n, const ot_options& o, Stream st) {
  require(src != nullptr, "input array is NULL");
  if (o.memspace == OT_MEM_HOST)
    dev::copy_h2d(dst, src, sizeof(double) * (size_t)n, st);
  else
    dev::copy_d2d(dst, src, sizeof(double) * (size_t)n, st);
}

static void copy_out(double* dst, const double* src, i64 n, const ot_options& o, Stream st) {
  if (!dst) return;
  if (o.memspace == OT_MEM_HOST)
    dev::copy_d2h(dst, src, sizeof(double) * (size_t)n, st);
  else
    dev::copy_d2d(dst, src, sizeof(double) * (size_t)n, st);
}

// rho_in, rho_f: finite, >= 0, positive sum per cell, equal masses (Sec. 2.2, Remark one-mass).
static void check_boundary_densities(const ot_mesh* m, const double* r0, const double* r1, const ot_options& o,
                                     Stream st) {
  require(r0 && r1, "rho_in / rho_f is NULL");
  i64 Nc = 2LL * m->n * m->n;
  std::vector<double> a(Nc), b(Nc);
  if (o.memspace == OT_MEM_HOST) {
    std::memcpy(a.data(), r0, sizeof(double) * Nc);
    std::memcpy(b.data(), r1, sizeof(double) * Nc);
  } else {
    dev::copy_d2h(a.data(), r0, sizeof(double) * Nc, st);
    dev::copy_d2h(b.data(), r1, sizeof(double) * Nc, st);
    dev::sync(st);
  }
  double ma = 0.0, mb = 0.0;
  for (i64 i = 0; i < Nc; ++i) {
    if (!isfinite(a[i]) || !isfinite(b[i])) throw Error(OT_ERR_NONFINITE, "rho_in / rho_f contain NaN or Inf");
    if (a[i] < 0 || b[i] < 0) throw Error(OT_ERR_NEGATIVE_DENSITY, "rho_in / rho_f must be >= 0");
    if (!(a[i] + b[i] > 0))
      throw Error(OT_ERR_NEGATIVE_DENSITY, "rho_in + rho_f must be > 0 in every cell (initial point needs rho > 0)");
    ma += a[i];
    mb += b[i];
  }
  if (!(ma > 0)) throw Error(OT_ERR_NEGATIVE_DENSITY, "rho_in has zero mass");
  if (fabs(ma - mb) > 1e-12 * std::max(ma, mb)) throw Error(OT_ERR_MASS_MISMATCH, "rho_in and rho_f masses differ");
}

// Copy (phi, rho, s, rho_in, rho_f) into the workspace.
static void load_state(Workspace& W, const double* phi, const double* rho, const double* s, const double* r0,
                       const double* r1, const ot_options& o, Stream st) {
  copy_in(W.phi, phi, W.Np, o, st);
  copy_in(W.rho, rho, W.Nr, o, st);
  copy_in(W.s, s, W.Nr, o, st);
  copy_in(W.r0, r0, W.d.Nc, o, st);
  copy_in(W.r1, r1, W.d.Nc, o, st);
}

static void require_positive(Workspace& W, const double* x, i64 n, const char* what, Stream st) {
  ot::k_min(x, n, W.scal + 40, W.partial, st);
  dev::copy_d2h(W.host, W.scal + 40, sizeof(double), st);
  dev::sync(st);
  if (!(W.host[0] > 0)) throw Error(OT_ERR_NEGATIVE_DENSITY, std::string(what) + " must be > 0");
}

static void gauge_phi(Workspace& W, double* phi, Stream st) {
  ot::k_slice_sums(phi, 1, W.Np, 1.0 / (double)W.Np, W.scal + 48, st);
  ot::k_slice_shift(phi, 1, W.Np, W.scal + 48, 1.0, st);
}

extern "C" {

ot_status ot_mesh_create(const ot_mesh_desc* desc, ot_mesh** out) {
  OT_TRY
  require(desc && out, "NULL argument");
  require(desc->kind == OT_MESH_STRUCTURED_SQUARE || desc->kind == OT_MESH_CARTESIAN_CUBE, "unsupported mesh kind");
  if (desc->kind == OT_MESH_STRUCTURED_SQUARE)
    require(supported_side(desc->n), "n must be 2^a * b with b <= 11 and n <= 4096");
  else
    require(desc->n >= 1 && desc->n <= 1024, "cube grids need 1 <= n <= 1024");
  ot_mesh* m = new ot_mesh();
  m->kind = desc->kind;
  m->n = desc->n;
  *out = m;
  return OT_OK;
  OT_CATCH
}

void ot_mesh_destroy(ot_mesh* mesh) { delete mesh; }

ot_status ot_mesh_info(const ot_mesh* mesh, int64_t* n_coarse, int64_t* n_fine, int64_t* n_edges_fine,
                       double* coarse_areas) {
  OT_TRY
  require(mesh != nullptr, "mesh is NULL");
  i64 n = mesh->n, m = 2 * n;
  if (is_cube(mesh)) {  // one grid of n^3 cubes, 3 n^2 (n - 1) interior faces
    if (n_coarse) *n_coarse = n * n * n;
    if (n_fine) *n_fine = n * n * n;
    if (n_edges_fine) *n_edges_fine = 3 * n * n * (n - 1);
    if (coarse_areas)
      for (i64 i = 0; i < n * n * n; ++i) coarse_areas[i] = 1.0 / (double)(n * n * n);
    return OT_OK;
  }
  if (n_coarse) *n_coarse = 2 * n * n;
  if (n_fine) *n_fine = 2 * m * m;
  if (n_edges_fine) *n_edges_fine = 3 * m * m - 2 * m;
  if (coarse_areas)
    for (i64 i = 0; i < 2 * n * n; ++i) coarse_areas[i] = 0.5 / (double)(n * n);
  return OT_OK;
  OT_CATCH
}

// One interior-point solve in the workspace W (sized for the mesh and K).
static void solve_in(Workspace& W, const ot_mesh* mesh, const double* rho_in, const double* rho_f, double mu0,
                     double tol, const ot_options& o, int32_t warm_start, double* rho, double* phi, double* s,
                     double* cost, ot_stats* stats, Stream st) {
  require(mu0 > 0 && tol > 0, "mu0 and tol must be positive");
  require(rho && phi && s, "output arrays are NULL");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  check_boundary_densities(mesh, rho_in, rho_f, o, st);
  copy_in(W.r0, rho_in, W.d.Nc, o, st);
  copy_in(W.r1, rho_f, W.d.Nc, o, st);
  if (warm_start) {
    copy_in(W.phi, phi, W.Np, o, st);
    copy_in(W.rho, rho, W.Nr, o, st);
    copy_in(W.s, s, W.Nr, o, st);
    require_positive(W, W.rho, W.Nr, "warm-start rho", st);
    require_positive(W, W.s, W.Nr, "warm-start s", st);
  } else {
    ot::k_init_point(W.d, mu0, W.r0, W.r1, W.phi, W.rho, W.s, st);
  }
  ot::ipm_run(W, o, mu0, tol, stats, st);
  gauge_phi(W, W.phi, st);
  ot::k_cost_dual(W.d, W.phi, W.rho, W.r0, W.r1, W.scal + 56, W.partial, st);
  dev::copy_d2h(W.host, W.scal + 56, 2 * sizeof(double), st);
  copy_out(rho, W.rho, W.Nr, o, st);
  copy_out(phi, W.phi, W.Np, o, st);
  copy_out(s, W.s, W.Nr, o, st);
  dev::sync(st);
  if (cost) *cost = W.host[0];
  if (stats) {
    stats->cost = W.host[0];
    stats->dual = W.host[1];
  }
}

ot_status ot_ipm_solve(ot_mesh* mesh, const double* rho_in, const double* rho_f, int32_t K, double mu0, double tol,
                       const ot_options* opt_in, int32_t warm_start, double* rho, double* phi, double* s,
                       double* cost, ot_stats* stats, void* cuda_stream) {
  OT_TRY
  ot_options o = resolve(opt_in);
  require(mesh != nullptr, "mesh is NULL");
  // checks that need no device memory come before the workspace is allocated
  require(mu0 > 0 && tol > 0, "mu0 and tol must be positive");
  require(rho_in && rho_f, "rho_in / rho_f is NULL");
  require(rho && phi && s, "output arrays are NULL");
  Workspace& W = workspace(mesh, K, o);
  solve_in(W, mesh, rho_in, rho_f, mu0, tol, o, warm_start, rho, phi, s, cost, stats, cuda_stream);
  return OT_OK;
  OT_CATCH
}

ot_status ot_ipm_solve_batched(int32_t n_prob, ot_mesh* const* meshes, const int32_t* K, const double* const* rho_in,
                               const double* const* rho_f, double mu0, double tol, const ot_options* opt_in,
                               double* const* rho, double* const* phi, double* const* s, double* cost,
                               ot_stats* stats, int32_t* status, int32_t n_streams) {
  OT_TRY
  ot_options o = resolve(opt_in);
  require(n_prob >= 0, "n_prob must be >= 0");
  require(n_streams >= 1 && n_streams <= 64, "n_streams must be in [1, 64]");
  if (n_prob == 0) return OT_OK;
  require(meshes && K && rho_in && rho_f && rho && phi && s, "NULL argument");
  for (int p = 0; p < n_prob; ++p) {
    require(meshes[p] != nullptr, "a mesh is NULL");
    require(K[p] >= 1 && K[p] <= 4096, "K must be in [1, 4096]");
  }
  const int device = dev::current_device();
  // largest problems first, so that the last ones to start are the short ones
  std::vector<int> order(n_prob);
  for (int p = 0; p < n_prob; ++p) order[p] = p;
  auto work = [&](int p) { return (double)meshes[p]->n * meshes[p]->n * (K[p] + 1.0); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work(a) > work(b); });
  std::atomic<int> next{0};
  std::vector<int> codes(n_prob, OT_OK);
  std::vector<std::string> msgs(n_prob);
  // the streams share one Krylov memory budget
  const size_t budget = ((size_t)96 << 30) / (size_t)std::min<int>(n_streams, n_prob);
  auto worker = [&]() {
    ot::prof::suspended = true;
    dev::set_krylov_budget(budget);
    Stream stream = nullptr;
    try {
      dev::set_device(device);
      stream = dev::stream_create();
      dev::set_alloc_stream(stream);
    } catch (const std::exception& e) {
      for (int i; (i = next.fetch_add(1)) < n_prob;) codes[order[i]] = OT_ERR_CUDA, msgs[order[i]] = e.what();
      return;
    }
    // this thread's workspace, replaced when the next problem's (side, K) differs
    std::map<std::pair<int, int>, std::unique_ptr<Workspace>> mine;
    for (int i; (i = next.fetch_add(1)) < n_prob;) {
      const int p = order[i];
      try {
        auto key = std::make_pair(meshes[p]->n, (int)K[p]);
        auto it = mine.find(key);
        if (it == mine.end()) {
          mine.clear();
          it = mine.emplace(key, std::unique_ptr<Workspace>(new Workspace(meshes[p]->n, K[p], o.precision, o))).first;
        }
        solve_in(*it->second, meshes[p], rho_in[p], rho_f[p], mu0, tol, o, 0, rho[p], phi[p], s[p],
                 cost ? cost + p : nullptr, stats ? stats + p : nullptr, stream);
      } catch (const ot::Error& e) {
        codes[p] = e.code, msgs[p] = e.what();
      } catch (const std::bad_alloc&) {
        codes[p] = OT_ERR_OOM, msgs[p] = "host allocation failed";
      } catch (const std::exception& e) {
        codes[p] = OT_ERR_CUDA, msgs[p] = e.what();
      }
    }
    dev::sync_quiet(stream);
    mine.clear();
    dev::sync_quiet(stream);
    dev::set_alloc_stream(nullptr);
    dev::stream_destroy(stream);
  };
  const int nt = std::min<int>(n_streams, n_prob);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& t : pool) t.join();
  int first = -1;
  for (int p = 0; p < n_prob; ++p) {
    if (status) status[p] = codes[p];
    if (codes[p] != OT_OK && first < 0) first = p;
  }
  if (first >= 0) throw Error(codes[first], "problem " + std::to_string(first) + ": " + msgs[first]);
  return OT_OK;
  OT_CATCH
}

ot_status ot_newton_solve(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho,
                          const double* s, const double* rho_in, const double* rho_f, const ot_options* opt_in,
                          double* dphi, double* drho, double* ds, ot_stats* stats, void* cuda_stream) {
  OT_TRY
  ot_options o = resolve(opt_in);
  require(mu > 0, "mu must be positive");
  Stream st = cuda_stream;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  Workspace& W = workspace(mesh, K, o);
  load_state(W, phi, rho, s, rho_in, rho_f, o, st);
  require_positive(W, W.rho, W.Nr, "rho", st);
  require_positive(W, W.s, W.Nr, "s", st);
  W.outer_iters = W.inner_iters = W.capped_solves = 0;
  W.mu = mu;
  double t0 = dev::now();
  double f = ot::residual_norm(W, mu, st, nullptr);
  double eps = o.final_eps_out > 0 ? o.final_eps_out : o.eps_out;
  ot::newton_direction(W, o, f, eps, st);
  copy_out(dphi, W.sol, W.Np, o, st);
  copy_out(drho, W.sol + W.Np, W.Nr, o, st);
  copy_out(ds, W.ds, W.Nr, o, st);
  dev::sync(st);
  if (stats) {
    stats->newton_steps = 1;
    stats->fgmres_iters = W.outer_iters;
    stats->inner_iters = W.inner_iters;
    stats->final_residual = f;
    stats->mu = mu;
    stats->seconds = dev::now() - t0;
  }
  return OT_OK;
  OT_CATCH
}

ot_status ot_cost_grad(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho, const double* s,
                       const double* rho_in, const double* rho_f, const ot_options* opt_in, double* grad_in,
                       double* grad_f, void* cuda_stream) {
  OT_TRY
  ot_options o = resolve(opt_in);
  require(mu > 0, "mu must be positive");
  require(grad_in && grad_f, "output arrays are NULL");
  Stream st = cuda_stream;
  Workspace& W = workspace(mesh, K, o);
  load_state(W, phi, rho, s, rho_in, rho_f, o, st);
  require_positive(W, W.rho, W.Nr, "rho", st);
  require_positive(W, W.s, W.Nr, "s", st);
  W.mu = mu;
  // J^T lambda = dC/du reduces (eliminating lambda_s) to the symmetric saddle system (Sec. 3.1)
  ot::k_adjoint_rhs(W.d, W.phi, W.rho, W.r0, W.r1, W.rhs, W.gsum, st);
  ot::refresh_coefficients(W, st);
  // tolerance relative to |rhs| (squared norm left in device memory for the solver)
  ot::k_dot(W.rhs, W.rhs, W.ntot, W.scal + 40, W.partial, st);
  double eps = o.final_eps_out > 0 ? o.final_eps_out : o.eps_out;
  ot::fgmres(W, o, W.rhs, W.sol, eps, W.scal + 40, 1, st);
  ot::recover_direction(W, st);
  ot::k_adjoint_grad(W.d, W.phi, W.sol, W.u, W.u + W.d.Nc, st);
  // area gauge: the component along |c'| removed from each gradient (all |c'| are equal on
  // this mesh, so that is the mean of each of the two N'-vectors)
  ot::k_slice_sums(W.u, 2, W.d.Nc, 1.0 / (double)W.d.Nc, W.scal + 48, st);
  ot::k_slice_shift(W.u, 2, W.d.Nc, W.scal + 48, 1.0, st);
  copy_out(grad_in, W.u, W.d.Nc, o, st);
  copy_out(grad_f, W.u + W.d.Nc, W.d.Nc, o, st);
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

// ------------------------------------------------------------------ autotuner
ot_status ot_tune_newton(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho, const double* s,
                         const double* rho_in, const double* rho_f, ot_options* opt, int32_t n_cand,
                         const int32_t* cand, double* seconds, void* cuda_stream) {
  OT_TRY
  require(opt != nullptr, "opt is NULL");
  const ot_options base = resolve(opt);
  require(mesh != nullptr, "mesh is NULL");
  require(mu > 0, "mu must be positive");
  require(phi && rho && s && rho_in && rho_f, "NULL argument");
  std::vector<int32_t> grid;  // (smooth_sweeps, coarse_sweeps, lap_cycles) per candidate
  if (cand) {
    require(n_cand >= 1 && n_cand <= 1024, "n_cand must be in [1, 1024]");
    grid.assign(cand, cand + 3 * (size_t)n_cand);
  } else {
    for (int sw = 1; sw <= 3; ++sw)
      for (int cs : {6, 10})
        for (int lc = 1; lc <= 2; ++lc) grid.insert(grid.end(), {sw, cs, lc});
  }
  const int nc = (int)(grid.size() / 3);
  auto with = [&](int i) {
    ot_options t = base;
    t.smooth_sweeps = grid[3 * i];
    t.coarse_sweeps = grid[3 * i + 1];
    t.lap_cycles = grid[3 * i + 2];
    return t;
  };
  for (int i = 0; i < nc; ++i) {  // every candidate must be a valid setting
    const ot_options t = with(i);
    resolve(&t);
  }
  ot_stats st;
  // untimed first solve: workspace allocation and first-touch costs stay out of the trials
  ot_status r = ot_newton_solve(mesh, K, mu, phi, rho, s, rho_in, rho_f, &base, nullptr, nullptr, nullptr, &st,
                                cuda_stream);
  if (r != OT_OK) return r;
  int best = -1;
  double tbest = 0.0;
  ot_status err = OT_OK;
  std::string msg;
  for (int i = 0; i < nc; ++i) {
    const ot_options t = with(i);
    const double t0 = dev::now();
    r = ot_newton_solve(mesh, K, mu, phi, rho, s, rho_in, rho_f, &t, nullptr, nullptr, nullptr, &st, cuda_stream);
    const double el = dev::now() - t0;
    if (r == OT_OK && st.fgmres_iters >= t.fgmres_max_iter) {  // capped: not a usable setting
      r = OT_ERR_NOT_CONVERGED;
      g_err = "FGMRES reached its iteration cap";
    }
    if (seconds) seconds[i] = r == OT_OK ? el : -1.0;
    if (r != OT_OK) {
      if (err == OT_OK) err = r, msg = g_err;
      continue;
    }
    if (best < 0 || el < tbest) best = i, tbest = el;
  }
  if (best < 0) return set_err(err, "every candidate failed; first: " + msg);
  opt->smooth_sweeps = grid[3 * best];
  opt->coarse_sweeps = grid[3 * best + 1];
  opt->lap_cycles = grid[3 * best + 2];
  g_err.clear();
  return OT_OK;
  OT_CATCH
}

// ------------------------------------------------------------------ operator-level entry points
// Any cached workspace of this K serves as scratch for the operator-level calls.
static Workspace& op_workspace(ot_mesh* mesh, int K) {
  require(mesh != nullptr, "mesh is NULL");
  require(!is_cube(mesh), "3D Cartesian meshes support only ot_residual, ot_kkt_apply and ot_cost_dual");
  for (auto& kv : mesh->ws)
    if (kv.first.first == K) return *kv.second;
  ot_options o;
  ot_default_options(&o);
  return workspace(mesh, K, o);
}

ot_status ot_residual(ot_mesh* mesh, int32_t K, double mu, const double* phi, const double* rho, const double* s,
                      const double* rho_in, const double* rho_f, double* F_phi, double* F_rho, double* F_s,
                      double* norms, void* cuda_stream) {
  OT_TRY
  require(mesh && phi && rho && s && rho_in && rho_f && F_phi && F_rho && F_s, "NULL argument");
  Stream st = cuda_stream;
  if (is_cube(mesh)) {
    require(K >= 1 && K <= 4096, "K must be in [1, 4096]");
    const ot::CubeDims d = ot::make_cube_dims(mesh->n, K);
    ot::k_cube_residual(d, mu, phi, rho, s, rho_in, rho_f, F_phi, F_rho, F_s, st);
    if (norms) {
      CubeScratch sc(8 + ot::k_reduce_scratch(1));
      ot::k_dot(F_phi, F_phi, (i64)(K + 1) * d.N, sc.dev + 0, sc.dev + 8, st);
      ot::k_dot(F_rho, F_rho, (i64)K * d.N, sc.dev + 1, sc.dev + 8, st);
      ot::k_dot(F_s, F_s, (i64)K * d.N, sc.dev + 2, sc.dev + 8, st);
      double h3[3];
      dev::copy_d2h(h3, sc.dev, 3 * sizeof(double), st);
      dev::sync(st);
      for (int i = 0; i < 3; ++i) norms[i] = sqrt(h3[i]);
      norms[3] = sqrt(h3[0] + h3[1] + h3[2]);
    }
    dev::sync(st);
    return OT_OK;
  }
  Workspace& W = op_workspace(mesh, K);
  ot::k_residual(W.d, mu, phi, rho, s, rho_in, rho_f, F_phi, F_rho, F_s, st);
  if (norms) {
    ot::k_dot(F_phi, F_phi, W.Np, W.scal + 0, W.partial, st);
    ot::k_dot(F_rho, F_rho, W.Nr, W.scal + 1, W.partial, st);
    ot::k_dot(F_s, F_s, W.Nr, W.scal + 2, W.partial, st);
    dev::copy_d2h(W.host, W.scal, 3 * sizeof(double), st);
  }
  dev::sync(st);
  if (norms) {
    for (int i = 0; i < 3; ++i) norms[i] = sqrt(W.host[i]);
    norms[3] = sqrt(W.host[0] + W.host[1] + W.host[2]);
  }
  return OT_OK;
  OT_CATCH
}

ot_status ot_kkt_apply(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* s,
                       const double* rho_in, const double* rho_f, const double* x, double* y, void* cuda_stream) {
  OT_TRY
  require(mesh && phi && rho && s && rho_in && rho_f && x && y, "NULL argument");
  Stream st = cuda_stream;
  if (is_cube(mesh)) {
    require(K >= 1 && K <= 4096, "K must be in [1, 4096]");
    CubeScratch sc(2 * (size_t)K + 2);
    ot::k_cube_kkt_apply(ot::make_cube_dims(mesh->n, K), phi, rho, s, rho_in, rho_f, x, y, sc.dev, st);
    dev::sync(st);
    return OT_OK;
  }
  Workspace& W = op_workspace(mesh, K);
  ot::k_kkt_coef(W.d, phi, rho, s, rho_in, rho_f, W.kcoef, st);
  ot::k_kkt_apply(W.d, W.kcoef, x, y, W.xmean, nullptr, st);
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

ot_status ot_kkt_apply_noalloc(int32_t n, int32_t K, const double* phi, const double* rho, const double* s,
                               const double* rho_in, const double* rho_f, const double* x, double* y,
                               void* cuda_stream) {
  OT_TRY
  require(supported_side(n), "n must be 2^a * b with b <= 11 and n <= 4096");
  require(K >= 1, "K must be >= 1");
  require(K <= ot::kStaticKktMaxK, "K exceeds the no-allocation limit (4096 slices)");
  require(phi && rho && s && rho_in && rho_f && x && y, "NULL argument");
  Stream st = cuda_stream;
  ot::k_kkt_apply_static(ot::make_dims(n, K), phi, rho, s, rho_in, rho_f, x, y, st);
  dev::check("ot_kkt_apply_noalloc launch");
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

ot_status ot_schur_apply(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* s,
                         const double* z, double* out, void* cuda_stream) {
  OT_TRY
  require(mesh && phi && rho && s && z && out, "NULL argument");
  Stream st = cuda_stream;
  Workspace& W = op_workspace(mesh, K);
  ot::k_schur_apply(W.d, phi, rho, s, z, out, W.u, st);
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

ot_status ot_simple_apply(ot_mesh* mesh, int32_t K, const ot_options* opt_in, const double* phi, const double* rho,
                          const double* s, const double* rho_in, const double* rho_f, const double* v, double* out,
                          void* cuda_stream) {
  OT_TRY
  ot_options o = resolve(opt_in);
  o.memspace = OT_MEM_DEVICE;
  require(v && out, "NULL argument");
  Stream st = cuda_stream;
  Workspace& W = workspace(mesh, K, o);
  load_state(W, phi, rho, s, rho_in, rho_f, o, st);
  ot::refresh_coefficients(W, st);
  ot::simple_prepare(W, st);
  ot::simple_apply(W, o, v, out, st);
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

ot_status ot_bb_apply(ot_mesh* mesh, int32_t K, const ot_options* opt_in, const double* phi, const double* rho,
                      const double* s, const double* rho_in, const double* rho_f, const double* v, double* out,
                      void* cuda_stream) {
  OT_TRY
  ot_options o = resolve(opt_in);
  o.memspace = OT_MEM_DEVICE;
  require(v && out, "NULL argument");
  Stream st = cuda_stream;
  Workspace& W = workspace(mesh, K, o);
  load_state(W, phi, rho, s, rho_in, rho_f, o, st);
  ot::refresh_coefficients(W, st);
  ot::bb_apply(W, o, v, out, st);
  dev::sync(st);
  return OT_OK;
  OT_CATCH
}

void ot_kernel_timing_enable(int32_t group_mask, int32_t sample_every) {
  ot::prof::reset();
  ot::prof::mask = (unsigned)group_mask;
  ot::prof::stride = sample_every > 1 ? sample_every : 1;
  ot::prof::enabled = group_mask != 0;
}

int32_t ot_kernel_timing_count(void) { return ot::prof::COUNT; }

int64_t ot_kernel_launches(void) { return ot::prof::n_launch; }

ot_status ot_kernel_timing_read(int32_t i, const char** name, double* ms, int64_t* launches, double* bytes) {
  OT_TRY
  require(i >= 0 && i < ot::prof::COUNT, "kernel group index out of range");
  double m = 0, b = 0;
  long long n = 0;
  ot::prof::read(i, &m, &n, &b);
  if (name) *name = ot::prof::name(i);
  if (ms) *ms = m;
  if (launches) *launches = n;
  if (bytes) *bytes = b;
  return OT_OK;
  OT_CATCH
}

ot_status ot_cost_dual(ot_mesh* mesh, int32_t K, const double* phi, const double* rho, const double* rho_in,
                       const double* rho_f, double* cost, double* dual, void* cuda_stream) {
  OT_TRY
  require(mesh && phi && rho && rho_in && rho_f, "NULL argument");
  Stream st = cuda_stream;
  if (is_cube(mesh)) {
    require(K >= 1 && K <= 4096, "K must be in [1, 4096]");
    const ot::CubeDims d = ot::make_cube_dims(mesh->n, K);
    CubeScratch sc(2 * (size_t)d.N + 2);
    ot::k_cube_cost_dual(d, phi, rho, rho_in, rho_f, sc.dev + 2 * d.N, sc.dev, st);
    dev::copy_d2h(sc.host, sc.dev + 2 * d.N, 2 * sizeof(double), st);
    dev::sync(st);
    if (cost) *cost = sc.host[0];
    if (dual) *dual = sc.host[1];
    return OT_OK;
  }
  Workspace& W = op_workspace(mesh, K);
  ot::k_cost_dual(W.d, phi, rho, rho_in, rho_f, W.scal + 56, W.partial, st);
  dev::copy_d2h(W.host, W.scal + 56, 2 * sizeof(double), st);
  dev::sync(st);
  if (cost) *cost = W.host[0];
  if (dual) *dual = W.host[1];
  return OT_OK;
  OT_CATCH
}

}  // extern "C"
