// solver.cpp -- host orchestration: multigrid cycles, (F)GMRES, the BB
// preconditioner, Newton directions and the interior-point loop.  Plain C++:
// device work goes through the launchers of ot_internal.h.
#include "solver.h"

#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

namespace ot {

// ------------------------------------------------------------------ storage
template <typename T>
void Hierarchy<T>::build(int m0, int S_, bool tc) {
  release();
  S = S_;
  time_coupled = tc;
  int m = m0;
  while (true) {
    LevelView<T> L;
    L.m = m;
    L.nc = 2LL * m * m;
    L.ld = L.nc;
    size_t v = sizeof(T) * (size_t)S * L.nc;
    L.alpha = (T*)dev::alloc(3 * v);
    L.tau = tc ? (T*)dev::alloc(v) : nullptr;
    L.x = (T*)dev::alloc(v);
    L.b = (T*)dev::alloc(v);
    L.r = (T*)dev::alloc(v);
    L.fac = tc ? (T*)dev::alloc(2 * v) : nullptr;
    lv.push_back(L);
    if (m % 2 != 0 || m == 1) break;
    m /= 2;
  }
  size_t v0 = sizeof(T) * (size_t)S * lv[0].nc;
  if (tc) {
    line_c = (T*)dev::alloc(v0);
    line_r = (T*)dev::alloc(v0);
  }
  agg = (T*)dev::alloc(sizeof(T) * 4 * (size_t)S);
  acc = (T*)dev::alloc(v0);
  bsave = (T*)dev::alloc(v0);
  // small levels run fused in one launch from shared memory: per-slice CTAs up
  // to side 32 for the slice Laplacians, one CTA up to side 8 for the
  // space-time operator (K <= 128); the largest such tail that fits.
  const int fuse_side = tc ? 8 : 32;
  fuse_from = lv.size();
  if (!tc || S <= 128)
    for (size_t l = 0; l < lv.size(); ++l)
      if (lv[l].m <= fuse_side &&
          k_mg_fused_smem<T>(S, lv.data() + l, (int)(lv.size() - l)) <= kFusedSmemLimit) {
        fuse_from = l;
        break;
      }
  if (fuse_from < lv.size()) k_mg_prepare_lower_cycle<T>(S, lv.data() + fuse_from, (int)(lv.size() - fuse_from));
}

template <typename T>
void Hierarchy<T>::release() {
  for (auto& L : lv) {
    dev::release(L.alpha);
    dev::release(L.tau);
    dev::release(L.x);
    dev::release(L.b);
    dev::release(L.r);
    dev::release(L.fac);
  }
  lv.clear();
  dev::release(line_c);
  dev::release(line_r);
  dev::release(agg);
  dev::release(acc);
  dev::release(bsave);
  line_c = line_r = agg = acc = bsave = nullptr;
}

template struct Hierarchy<float>;
template struct Hierarchy<double>;

template <typename T>
void KrylovT<T>::build(int m, i64 n_, bool shadow) {
  release();
  mmax = m;
  n = n_;
  if (shadow) {
    V32 = (float*)dev::alloc(sizeof(float) * (size_t)(m + 1) * n);
    w32 = (float*)dev::alloc(sizeof(float) * (size_t)n);
  }
  V = (T*)dev::alloc(sizeof(T) * (size_t)(m + 1) * n);
  Z = (T*)dev::alloc(sizeof(T) * (size_t)m * n);
  w = (T*)dev::alloc(sizeof(T) * (size_t)n);
  in = (T*)dev::alloc(sizeof(T) * (size_t)n);
  zout = (T*)dev::alloc(sizeof(T) * (size_t)n);
  hc1 = (double*)dev::alloc(sizeof(double) * (m + 2));
  hc2 = (double*)dev::alloc(sizeof(double) * (m + 2));
  y = (double*)dev::alloc(sizeof(double) * (m + 2));
  ctl = (kry::Ctl*)dev::alloc(sizeof(kry::Ctl));
  H = (double*)dev::alloc(sizeof(double) * (size_t)(m + 1) * (size_t)m);
  cs = (double*)dev::alloc(sizeof(double) * (m + 1));
  sn = (double*)dev::alloc(sizeof(double) * (m + 1));
  g = (double*)dev::alloc(sizeof(double) * (m + 2));
  part = (double*)dev::alloc(sizeof(double) * kry_partial_doubles(m));
  dev::zero(part + kry_counter_offset(m), 64 * sizeof(double), nullptr);  // arrival counters
  scal = (double*)dev::alloc(sizeof(double) * 8);
  kry::Ctl c0;
  std::memset(&c0, 0, sizeof(c0));
  c0.status = kry::CONVERGED;
  dev::copy_h2d(ctl, &c0, sizeof(c0), nullptr);
  dev::sync(nullptr);
}

template <typename T>
void KrylovT<T>::release() {
  void* bufs[] = {V, Z, w, in, zout, hc1, hc2, y, V32, w32, ctl, H, cs, sn, g, part, scal};
  for (void* b : bufs) dev::release(b);
  V = Z = w = in = zout = nullptr;
  hc1 = hc2 = y = H = cs = sn = g = part = scal = nullptr;
  V32 = w32 = nullptr;
  ctl = nullptr;
}
template struct KrylovT<float>;
template struct KrylovT<double>;

static double* dalloc(i64 n) { return (double*)dev::alloc(sizeof(double) * (size_t)(n > 0 ? n : 1)); }

int effective_restart(const ot_options& opt, i64 ntot) {
  if (opt.fgmres_restart > 0) return opt.fgmres_restart;
  const i64 per_vector = ntot * (i64)(2 * sizeof(double) + sizeof(float));  // V, Z and the FP32 shadow of V
  const i64 fit = (i64)(dev::krylov_budget() / (size_t)(per_vector > 0 ? per_vector : 1));
  const i64 cap = std::min<i64>(opt.fgmres_max_iter, kMaxRestart);
  return (int)std::max<i64>(std::min<i64>(30, cap), std::min<i64>(cap, fit));
}

Workspace::Workspace(int n, int K, int prec, const ot_options& opt) {
  d = make_dims(n, K);
  precision = prec;
  Np = (i64)(K + 1) * d.N;
  Nr = (i64)K * d.Nc;
  ntot = Np + Nr;
  try {
    phi = dalloc(Np);
    rho = dalloc(Nr);
    s = dalloc(Nr);
    r0 = dalloc(d.Nc);
    r1 = dalloc(d.Nc);
    Fphi = dalloc(Np);
    Frho = dalloc(Nr);
    Fs = dalloc(Nr);
    rhs = dalloc(ntot);
    sol = dalloc(ntot);
    ytmp = dalloc(ntot);
    hvec = dalloc(Nr);
    ds = dalloc(Nr);
    gsum = dalloc(K + 2);
    wsum = dalloc(K + 2);
    cshift = dalloc(K + 2);
    xmean = dalloc(K + 2);
    mass = dalloc(K + 2);
    scal = dalloc(64 + 2 * (K + 2));
    kcoef = dalloc(kkt_coef_count(d));
    cur_restart = effective_restart(opt, ntot);
    int mm = std::max(cur_restart, opt.schur_max_iter) + 2;
    partial = dalloc((i64)k_reduce_scratch(mm < 64 ? 64 : mm));
    u = dalloc(Np);
    bphi = dalloc(Np);
    srhs = dalloc(Nr);
    zeta = dalloc(Nr);
    cur_inner = opt.schur_max_iter;
    outer.build(cur_restart, ntot, true);
    if (prec == OT_PREC_MIXED) {
      innerf.build(cur_inner, Nr);
      // phi, u, bphi: Np each; rho, s, srhs, zeta, y: Nr each; mean, sums: K+2 each
      const i64 nf = 3 * Np + 5 * Nr + 2 * (K + 2);
      f32 = (float*)dev::alloc(sizeof(float) * (size_t)nf);
      float* p = f32;
      auto take = [&](i64 len) {
        float* q = p;
        p += len;
        return q;
      };
      phif = take(Np);
      rhof = take(Nr);
      sf = take(Nr);
      bbf.phi = phif;
      bbf.rho = rhof;
      bbf.s = sf;
      bbf.u = take(Np);
      bbf.bphi = take(Np);
      bbf.srhs = take(Nr);
      bbf.zeta = take(Nr);
      bbf.y = take(Nr);
      bbf.mean = take(K + 2);
      bbf.sums = take(K + 2);
      bbf.K = &innerf;
      lapf.build(d.m, K + 1, false);
      schf.build(d.n, K, true);
    } else {
      inner.build(cur_inner, Nr);
      bbd.phi = phi;
      bbd.rho = rho;
      bbd.s = s;
      bbd.u = u;
      bbd.bphi = bphi;
      bbd.srhs = srhs;
      bbd.zeta = zeta;
      bbd.y = nullptr;
      bbd.mean = xmean;
      bbd.sums = scal + 64;
      bbd.K = &inner;
      lapd.build(d.m, K + 1, false);
      schd.build(d.n, K, true);
    }
    hoff = std::max(cur_restart, cur_inner) + 4;
    host = (double*)dev::host_alloc(sizeof(double) * (size_t)(2 * hoff + 64));
  } catch (...) {
    this->~Workspace();
    throw;
  }
}

Workspace::~Workspace() {
  double* bufs[] = {phi, rho, s, r0, r1, Fphi, Frho, Fs, rhs, sol, ytmp, hvec, ds, gsum, wsum, cshift, xmean,
                    mass, scal, partial, u, bphi, srhs, zeta, kcoef, sAd, sinv, se, skin, sG, slam};
  for (double* b : bufs) dev::release(b);
  sAd = sinv = se = skin = sG = slam = nullptr;
  dev::release(sstat);
  sstat = nullptr;
  phi = rho = s = r0 = r1 = Fphi = Frho = Fs = rhs = sol = ytmp = hvec = ds = nullptr;
  gsum = wsum = cshift = xmean = mass = scal = partial = u = bphi = srhs = zeta = kcoef = nullptr;
  outer.release();
  inner.release();
  innerf.release();
  dev::release(f32);
  f32 = phif = rhof = sf = nullptr;
  lapf.release();
  schf.release();
  lapd.release();
  schd.release();
  dev::host_release(host);
  host = nullptr;
}

// ------------------------------------------------------------------ multigrid
template <typename T>
static void vcycle(Hierarchy<T>& H, size_t l, int nu, int nuc, Stream st) {
  LevelView<T>& L = H.lv[l];
  if (l == H.fuse_from) {
    k_mg_lower_cycle<T>(H.S, H.lv.data() + l, (int)(H.lv.size() - l), nu, nuc, H.line_c, H.line_r, H.agg, st);
    return;
  }
  if (l + 1 == H.lv.size()) {
    k_mg_coarse_solve<T>(H.S, L, nuc, H.line_c, H.line_r, H.agg, st);
    return;
  }
  LevelView<T>& Lc = H.lv[l + 1];
  if (nu == 0) {
    dev::zero(L.x, sizeof(T) * (size_t)H.S * L.nc, st);
    k_mg_residual<T>(H.S, L, st);
    k_mg_restrict<T>(H.S, L, Lc, st);
    vcycle(H, l + 1, nu, nuc, st);
    k_mg_prolong<T>(H.S, Lc, L, st);
    return;
  }
  // pre-smoothing from x = 0: the first sweep reads no neighbour value
  k_mg_smooth_mode<T>(H.S, L, nullptr, 0, 1, H.line_c, H.line_r, st);
  k_mg_smooth<T>(H.S, L, 1, H.line_c, H.line_r, st);
  for (int i = 1; i < nu; ++i) {
    k_mg_smooth<T>(H.S, L, 0, H.line_c, H.line_r, st);
    k_mg_smooth<T>(H.S, L, 1, H.line_c, H.line_r, st);
  }
  k_mg_restrict_residual<T>(H.S, L, Lc, st);
  vcycle(H, l + 1, nu, nuc, st);
  // post-smoothing: the first sweep adds the coarse correction to the neighbours it reads
  k_mg_smooth_mode<T>(H.S, L, &Lc, 1, 2, H.line_c, H.line_r, st);
  k_mg_smooth<T>(H.S, L, 0, H.line_c, H.line_r, st);
  for (int i = 1; i < nu; ++i) {
    k_mg_smooth<T>(H.S, L, 1, H.line_c, H.line_r, st);
    k_mg_smooth<T>(H.S, L, 0, H.line_c, H.line_r, st);
  }
}

// x ~= M^{-1} b by `cycles` V-cycles from zero (x in FP64; b in FP64 or T; the cycle in T).
template <typename T, typename In>
static void mg_solve(Hierarchy<T>& H, const In* b, double* x, int cycles, int nu, int nuc, Stream st) {
  LevelView<T>& L = H.lv[0];
  i64 n = (i64)H.S * L.nc;
  size_t bytes = sizeof(T) * (size_t)n;
  if constexpr (std::is_same<In, T>::value)
    dev::copy_d2d(L.b, b, bytes, st);
  else
    k_mg_load<T>(b, 1.0, L.b, nullptr, n, st);
  if (cycles <= 1) {
    vcycle(H, 0, nu, nuc, st);
    k_mg_store<T>(L.x, x, n, st);
    return;
  }
  dev::copy_d2d(H.bsave, L.b, bytes, st);
  vcycle(H, 0, nu, nuc, st);
  dev::copy_d2d(H.acc, L.x, bytes, st);
  for (int c = 1; c < cycles; ++c) {
    dev::copy_d2d(L.x, H.acc, bytes, st);
    dev::copy_d2d(L.b, H.bsave, bytes, st);
    k_mg_residual<T>(H.S, L, st);
    dev::copy_d2d(L.b, L.r, bytes, st);
    vcycle(H, 0, nu, nuc, st);
    k_mg_axpy<T>(L.x, (T)1, H.acc, n, st);
  }
  k_mg_store<T>(H.acc, x, n, st);
}

// x ~= M^{-1} b by one V-cycle, b and x in T: level 0 works on b and x in place.
template <typename T>
static void mg_apply(Hierarchy<T>& H, const T* b, T* x, int nu, int nuc, Stream st) {
  struct Swap {
    LevelView<T>& L;
    T *b0, *x0;
    ~Swap() {
      L.b = b0;
      L.x = x0;
    }
  } guard{H.lv[0], H.lv[0].b, H.lv[0].x};
  H.lv[0].b = const_cast<T*>(b);  // read only
  H.lv[0].x = x;
  vcycle(H, 0, nu, nuc, st);
}

template <typename T>
static void refresh_t(Workspace& W, Hierarchy<T>& lap, Hierarchy<T>& sch, Stream st) {
  k_mg_lap_coef0<T>(W.d, W.rho, W.r0, W.r1, lap.lv[0].alpha, st);
  for (size_t l = 0; l + 1 < lap.lv.size(); ++l) k_mg_restrict_coef<T>(lap.S, lap.lv[l], lap.lv[l + 1], st);
  k_mg_schur_coef0<T>(W.d, W.phi, W.rho, W.s, sch.lv[0].alpha, sch.lv[0].tau, st);
  for (size_t l = 0; l + 1 < sch.lv.size(); ++l) k_mg_restrict_coef<T>(sch.S, sch.lv[l], sch.lv[l + 1], st);
  // time-line factors of the levels the tiled smoother sweeps (the fused levels factor their own)
  for (size_t l = 0; l < sch.lv.size() && l < sch.fuse_from; ++l) k_mg_line_factor<T>(sch.S, sch.lv[l], st);
}

void refresh_coefficients(Workspace& W, Stream st) {
  k_kkt_coef(W.d, W.phi, W.rho, W.s, W.r0, W.r1, W.kcoef, st);
  if (W.precision == OT_PREC_MIXED) {
    refresh_t(W, W.lapf, W.schf, st);
    k_convert(W.phi, W.phif, W.Np, 1.0, st);
    k_convert(W.rho, W.rhof, W.Nr, 1.0, st);
    k_convert(W.s, W.sf, W.Nr, 1.0, st);
  } else
    refresh_t(W, W.lapd, W.schd, st);
}

// ------------------------------------------------------------------ Arnoldi
template <typename T>
using OpFn = std::function<void(const T*, T*, Stream)>;

// One Arnoldi step of right-preconditioned (flexible) GMRES, enqueued on st:
// z_j = M^{-1} v_j (v_j is K.in), w = A z_j, classical Gram-Schmidt with one
// reorthogonalisation against v_0..v_j (the step count j is read by the kernels
// from K.ctl), the last block of the final update sums |w|^2 and takes the
// Givens step (least squares, status, j += 1, loop condition), then one kernel
// writes v_{j+1} = w/|w| (also to K.in) and stores z_j in Z: seven or eight
// launches besides M and A.  With an FP32 shadow of the basis (shadow) the dot
// products of the first pass, and of the second when fp32_reorth is set, are
// taken from it in FP32; every coefficient is applied to the FP64 basis and H
// records exactly the coefficients applied, so the Arnoldi relation A Z = V H
// holds to FP64 rounding whichever precision computed them.
// Second-pass coefficients from the shadow limit the orthogonality of V to
// ~1e-7, which moves the residual estimate by that relative amount: harmless
// for a target of 1e-5, so fgmres() asks for it only for targets >= 1e-8.  In
// that mode the second pass is applied from the shadow too, its combination
// formed in FP32: those coefficients are ~1e-7 of |w|, so the FP32 rounding of
// the correction (and of the coefficients H records) is ~1e-14 of |w|.
template <typename T>
static void arnoldi_step(KrylovT<T>& K, const OpFn<T>& prec, const OpFn<T>& op, bool shadow, bool fp32_reorth,
                         Stream st, CondHandle h, int j) {
  const i64 n = K.n;
  const int nv = j >= 0 ? j + 1 : -1;
  // the Givens step rides on the last update (its last block, once |w|^2 is summed)
  KryGivens gv;
  gv.ctl = K.ctl;
  gv.hc1 = K.hc1;
  gv.hc2 = K.hc2;
  gv.H = K.H;
  gv.ldh = K.ldh();
  gv.cs = K.cs;
  gv.sn = K.sn;
  gv.g = K.g;
  gv.h = h.h;
  gv.on = (int)h.on;
  prec(K.in, K.zout, st);
  op(K.zout, K.w, st);
  if constexpr (std::is_same<T, double>::value) shadow = shadow && K.V32 != nullptr;
  else shadow = false;  // FP32 bases have no shadow
  if (shadow) {
    k_convert(reinterpret_cast<const double*>(K.w), K.w32, n, 1.0, st);
    kry_dot<float>(K.V32, n, K.ctl, 1, K.mmax, K.w32, n, K.hc1, K.part, nv, st);
    if (fp32_reorth) {
      // second pass entirely from the shadow: dots, and the update formed in FP32
      kry_update<T>(K.V, n, K.ctl, 1, K.mmax, K.hc1, K.w, n, K.w32, nullptr, K.part, nv, st);
      kry_dot<float>(K.V32, n, K.ctl, 1, K.mmax, K.w32, n, K.hc2, K.part, nv, st);
      kry_update_shadow(K.V32, n, K.ctl, 1, K.mmax, K.hc2, reinterpret_cast<double*>(K.w), n, K.hc2, K.part, nv, st,
                        &gv);
    } else {
      kry_update<T>(K.V, n, K.ctl, 1, K.mmax, K.hc1, K.w, n, nullptr, nullptr, K.part, nv, st);
      kry_dot<T>(K.V, n, K.ctl, 1, K.mmax, K.w, n, K.hc2, K.part, nv, st);
      kry_update<T>(K.V, n, K.ctl, 1, K.mmax, K.hc2, K.w, n, nullptr, K.hc2, K.part, nv, st, &gv);
    }
  } else {
    kry_dot<T>(K.V, n, K.ctl, 1, K.mmax, K.w, n, K.hc1, K.part, nv, st);
    kry_update<T>(K.V, n, K.ctl, 1, K.mmax, K.hc1, K.w, n, nullptr, nullptr, K.part, nv, st);
    kry_dot<T>(K.V, n, K.ctl, 1, K.mmax, K.w, n, K.hc2, K.part, nv, st);
    kry_update<T>(K.V, n, K.ctl, 1, K.mmax, K.hc2, K.w, n, nullptr, K.hc2, K.part, nv, st, &gv);
  }
  // the Givens step advanced ctl->j: the new basis vector and the Z slot of this step are j - 1 + 1 and j - 1
  kry_next_basis<T>(K.w, K.hc2, K.ctl, -1, K.V, n, shadow ? K.V32 : nullptr, K.in, K.zout, K.Z, n, st);
}

// One (F)GMRES cycle on stream st: start vector r (in K.w on entry of the
// prologue: `start` enqueues r = b - A x into K.w), V_0 = r/|r|, Arnoldi steps
// until the Givens kernel stops them, then y = R^{-1} g and x += Z y.  The tolerance
// is either relative to |r| (tol_rel > 0) or already in K.ctl (kry_solve_init).
template <typename T>
static void gmres_cycle(KrylovT<T>& K, int m, double tol_rel, const std::function<void(Stream)>& start,
                        const OpFn<T>& prec, const OpFn<T>& op, bool shadow, bool fp32_reorth, T* x, Stream st) {
  const i64 n = K.n;
  auto prologue = [&](Stream s, CondHandle h) {
    start(s);
    k_dot(K.w, K.w, n, K.scal, K.part, s);
    kry_start(K.ctl, K.scal, m, tol_rel, K.g, h, s);
    kry_start_basis<T>(K.w, K.scal, K.V, shadow ? K.V32 : nullptr, K.in, n, s);
  };
  auto body = [&](Stream s, CondHandle h, int j) { arnoldi_step<T>(K, prec, op, shadow, fp32_reorth, s, h, j); };
  dev::device_while(st, K.ctl, prologue, body);
  kry_backsolve(K.ctl, K.H, K.ldh(), K.g, K.y, st);
  kry_combine<T>(K.Z, n, K.ctl, K.mmax, K.y, x, n, -1, st);
}

// ------------------------------------------------------------------ BB preconditioner
// Inner solve of the Schur system to relative tolerance eps_schur: GMRES
// preconditioned by one space-time V-cycle, vectors in T, x = 0 initially.
template <typename T>
static void inner_solve(Workspace& W, const ot_options& opt, Hierarchy<T>& sch, const BBVectors<T>& B, const T* b,
                        T* x, Stream st) {
  KrylovT<T>& K = *B.K;
  const i64 n = W.Nr;
  const int m = std::min(opt.schur_max_iter, K.mmax);
  dev::zero(x, sizeof(T) * (size_t)n, st);
  OpFn<T> prec = [&](const T* in, T* out, Stream s) {
    mg_apply(sch, in, out, opt.smooth_sweeps, opt.coarse_sweeps, s);
  };
  OpFn<T> op = [&](const T* in, T* out, Stream s) { k_schur_apply(W.d, B.phi, B.rho, B.s, in, out, B.u, s); };
  auto start = [&](Stream s) {
    kry_solve_init(K.ctl, nullptr, 0, 0.0, m, s);
    dev::copy_d2d(K.w, b, sizeof(T) * (size_t)n, s);
  };
  gmres_cycle<T>(K, m, opt.eps_schur, start, prec, op, false, false, x, st);
}

// out = P_BB^{-1} v with v = (c; d) and out = (x; y) in FP64; the solves in T.
template <typename T>
static void bb_apply_t(Workspace& W, const ot_options& opt, Hierarchy<T>& lap, Hierarchy<T>& sch,
                       const BBVectors<T>& B, const double* v, double* out, Stream st) {
  constexpr bool f64 = std::is_same<T, double>::value;
  const Dims& d = W.d;
  const double* c = v;
  const double* dv = v + W.Np;
  double* x = out;
  double* y = out + W.Np;
  // Schur system (Eq. pseudoschur-bis): (Diag(s) A~ - Diag(rho) B M^-1 B~) z = -Diag(rho) d
  k_mul(B.rho, dv, -1.0, B.srhs, W.Nr, st);
  inner_solve(W, opt, sch, B, B.srhs, B.zeta, st);
  // y = M'^{-1} A~ z
  T* yt = nullptr;
  if constexpr (f64)
    yt = y;
  else
    yt = B.y;
  k_atilde_minv(d, B.rho, B.zeta, yt, st);
  if constexpr (!f64) k_convert(yt, y, W.Nr, 1.0, st);
  // b = c - B^T P^T y, kept in the range of A (zero slice sums)
  if constexpr (f64)
    k_bt_apply(d, W.kcoef, yt, B.bphi, B.mean, st);
  else
    k_bt_apply(d, B.phi, yt, B.bphi, B.mean, st);
  if constexpr (f64)
    k_axpby(1.0, c, -1.0, B.bphi, W.Np, st);
  else
    k_rsub(c, B.bphi, W.Np, st);
  k_slice_sums(B.bphi, d.K + 1, d.N, 1.0 / (double)d.N, B.sums, st);
  k_slice_shift(B.bphi, d.K + 1, d.N, B.sums, 1.0, st);
  // A^j x^j = b^j, j = 1..K+1, by multigrid (Eq. x-triang)
  mg_solve(lap, (const T*)B.bphi, x, opt.lap_cycles, opt.smooth_sweeps, opt.coarse_sweeps, st);
}

void bb_apply(Workspace& W, const ot_options& opt, const double* v, double* out, Stream st) {
  if (W.precision == OT_PREC_MIXED)
    bb_apply_t(W, opt, W.lapf, W.schf, W.bbf, v, out, st);
  else
    bb_apply_t(W, opt, W.lapd, W.schd, W.bbd, v, out, st);
}

// ------------------------------------------------------------------ SIMPLE
bool use_simple(const ot_options& opt, double mu) {
  return opt.precond == OT_PRECOND_SIMPLE || (opt.precond == OT_PRECOND_HYBRID && mu < opt.simple_mu);
}

void simple_prepare(Workspace& W, Stream st) {
  const Dims& d = W.d;
  if (d.K > kSimpleMaxK) throw Error(OT_ERR_INVALID_ARG, "the SIMPLE preconditioner needs K <= 1024");
  if (!W.sAd) {
    W.sAd = dalloc(W.Np);
    W.sinv = dalloc(W.Nr);
    W.se = dalloc(W.Nr);
    W.skin = dalloc(W.ntot);
    W.sG = dalloc((i64)d.K * d.K);
    W.slam = dalloc(2 * (i64)d.K);
    W.sstat = (int*)dev::alloc(sizeof(int));
  }
  if (!W.inner.ctl) W.inner.build(W.cur_inner, W.Nr);  // the FP64 inner Krylov space (mixed precision)
  k_simple_diag(d, W.kcoef, W.sAd, st);
  k_simple_line_factor(d, W.kcoef, W.sAd, W.sinv, W.se, st);
  dev::zero(W.sstat, sizeof(int), st);
  k_simple_gram(d, W.sinv, W.se, W.ytmp, W.sG, W.sstat, st);
  int bad = 0;
  dev::copy_d2h(&bad, W.sstat, sizeof(int), st);
  dev::sync(st);
  if (bad) throw Error(OT_ERR_BREAKDOWN, "SIMPLE: the slice-sum system of the time-line preconditioner is not positive definite");
}

// Sec. 4.2 with A^ = Diag(A) on the projected system [A, B^T P^T; P B, -P C P^T]:
//   x1 = A^-1 c;  solve -S^ y = P B x1 - d;  x = x1 - A^-1 B^T P^T y,
// -S^ = P C P^T + P B A^-1 B^T P^T applied through the KKT kernels: B^T P^T z,
// scaled by A^-1, enters the KKT operator with x_rho = -z, whose rho rows are then
// P B A^-1 B^T P^T z + P C P^T z.  The Krylov vectors stay in the range of P
// (zero slice sums); the preconditioner solves the time-line part exactly there.
void simple_apply(Workspace& W, const ot_options& opt, const double* v, double* out, Stream st) {
  const Dims& d = W.d;
  const i64 Np = W.Np, Nr = W.Nr;
  const double* c = v;
  const double* dv = v + Np;
  double* x = out;
  double* y = out + Np;
  double* kin = W.skin;
  double* kout = W.ytmp;
  // x1 = A^-1 c (kept in x); right-hand side P B x1 - d
  k_quot(c, W.sAd, 1.0, x, 0.0, Np, st);
  dev::copy_d2d(kin, x, sizeof(double) * (size_t)Np, st);
  dev::zero(kin + Np, sizeof(double) * (size_t)Nr, st);
  k_kkt_apply(d, W.kcoef, kin, kout, W.xmean, nullptr, st);
  dev::copy_d2d(W.srhs, kout + Np, sizeof(double) * (size_t)Nr, st);
  k_axpby(-1.0, dv, 1.0, W.srhs, Nr, st);
  // GMRES on -S^ y = P B x1 - d, preconditioned by the time-line solves
  KrylovT<double>& K = W.inner;
  const int m = std::min(opt.schur_max_iter, K.mmax);
  dev::zero(y, sizeof(double) * (size_t)Nr, st);
  // z = L^-1 (r - Y lambda) with (Y^T L^-1 Y) lambda = Y^T L^-1 r: P L P^T z = r, Y^T z = 0
  double* t = W.slam;
  double* lam = W.slam + d.K;
  OpFn<double> prec = [&](const double* in, double* o, Stream s) {
    k_simple_line_solve(d, W.sinv, W.se, in, nullptr, o, s);
    k_slice_sums(o, d.K, d.Nc, 1.0, t, s);
    k_simple_gram_solve(d.K, W.sG, t, lam, s);
    k_simple_line_solve(d, W.sinv, W.se, in, lam, o, s);
  };
  OpFn<double> op = [&](const double* in, double* o, Stream s) {
    k_bt_apply(d, W.kcoef, in, W.u, W.xmean, s);
    k_quot(W.u, W.sAd, 1.0, kin, 0.0, Np, s);
    k_scale(in, -1.0, kin + Np, Nr, s);
    k_kkt_apply(d, W.kcoef, kin, kout, W.xmean, nullptr, s);
    dev::copy_d2d(o, kout + Np, sizeof(double) * (size_t)Nr, s);
  };
  auto start = [&](Stream s) {
    kry_solve_init(K.ctl, nullptr, 0, 0.0, m, s);
    dev::copy_d2d(K.w, W.srhs, sizeof(double) * (size_t)Nr, s);
  };
  gmres_cycle<double>(K, m, opt.eps_schur, start, prec, op, false, false, y, st);
  // x = x1 - A^-1 B^T P^T y
  k_bt_apply(d, W.kcoef, y, W.u, W.xmean, st);
  k_quot(W.u, W.sAd, -1.0, x, 1.0, Np, st);
}

// ------------------------------------------------------------------ FGMRES
// Inner iterations so far (device counters of the inner solvers: the FP32 one of
// mixed-precision BB, the FP64 one of FP64 BB and of SIMPLE).
static long long inner_total(Workspace& W, Stream st) {
  long long t = 0;
  kry::Ctl c;
  if (W.innerf.ctl) {
    dev::read_ctl(W.innerf.ctl, &c, st);
    t += c.total;
  }
  if (W.inner.ctl) {
    dev::read_ctl(W.inner.ctl, &c, st);
    t += c.total;
  }
  return t;
}

double fgmres(Workspace& W, const ot_options& opt, const double* b, double* x, double tol_rel,
              const double* tol_ref, int nref, Stream st) {
  dev::PdlScope pdl_scope(opt.pdl != 0);
  Krylov& K = W.outer;
  const i64 n = W.ntot;
  const bool shadow = opt.gs_shadow && K.V32 != nullptr;
  const bool fp32_reorth = shadow && tol_rel >= 1e-8;
  const int m = std::min(effective_restart(opt, n), K.mmax);
  const bool simple = use_simple(opt, W.mu);
  if (simple) simple_prepare(W, st);
  OpFn<double> prec = [&](const double* in, double* out, Stream s) {
    if (simple)
      simple_apply(W, opt, in, out, s);
    else
      bb_apply(W, opt, in, out, s);
  };
  OpFn<double> op = [&](const double* in, double* out, Stream s) {
    k_kkt_apply(W.d, W.kcoef, in, out, W.xmean, nullptr, s);
  };
  dev::zero(x, sizeof(double) * (size_t)n, st);
  kry_solve_init(K.ctl, tol_ref, nref, tol_rel, opt.fgmres_max_iter, st);
  const long long inner0 = inner_total(W, st);
  kry::Ctl c;
  bool first = true;
  while (true) {
    // the first cycle starts from x = 0 (r = b), later ones from the true residual r = b - A x
    auto start = [&, first](Stream s) {
      if (first) {
        dev::copy_d2d(K.w, b, sizeof(double) * (size_t)n, s);
      } else {
        op(x, K.w, s);
        k_axpby(1.0, b, -1.0, K.w, n, s);
      }
    };
    if (opt.graphs) {
      char key[160];
      snprintf(key, sizeof(key), "fgmres:%d:%d:%d:%d:%d:%d:%d:%.17g:%p:%p:%p:%d:%d", (int)first, m, (int)shadow,
               (int)fp32_reorth, opt.smooth_sweeps, opt.coarse_sweeps, opt.lap_cycles, opt.eps_schur, (const void*)b,
               (const void*)x, (const void*)tol_ref, opt.schur_max_iter, (int)simple + 2 * (opt.pdl != 0));
      std::unique_ptr<dev::Graph>& gp = W.graphs[key];
      if (!gp) {
        gp.reset(new dev::Graph());
        gp->capture([&](Stream s) { gmres_cycle<double>(K, m, 0.0, start, prec, op, shadow, fp32_reorth, x, s); });
      }
      kry::Ctl before;
      dev::read_ctl(K.ctl, &before, st);
      const long long in_before = inner_total(W, st);
      gp->launch(st);
      dev::read_ctl(K.ctl, &c, st);
      const long long in_after = inner_total(W, st);
      prof::n_launch += gp->executed({c.total - before.total, in_after - in_before});
    } else {
      gmres_cycle<double>(K, m, 0.0, start, prec, op, shadow, fp32_reorth, x, st);
      dev::read_ctl(K.ctl, &c, st);
    }
    if (c.status == kry::NONFINITE) throw Error(OT_ERR_NONFINITE, "non-finite value in the Krylov iteration");
    if (c.status != kry::LIMIT || c.base >= c.cap) break;
    first = false;
  }
  W.outer_iters += c.base;
  W.inner_iters += inner_total(W, st) - inner0;
  if (c.res > c.tol) W.capped_solves++;
  return c.res;
}

// ------------------------------------------------------------------ Newton
double residual_norm(Workspace& W, double mu, Stream st, double* norms) {
  k_residual(W.d, mu, W.phi, W.rho, W.s, W.r0, W.r1, W.Fphi, W.Frho, W.Fs, st);
  k_dot(W.Fphi, W.Fphi, W.Np, W.scal + 0, W.partial, st);
  k_dot(W.Frho, W.Frho, W.Nr, W.scal + 1, W.partial, st);
  k_dot(W.Fs, W.Fs, W.Nr, W.scal + 2, W.partial, st);
  dev::copy_d2h(W.host, W.scal, 3 * sizeof(double), st);
  dev::sync(st);
  double t = 0.0;
  for (int i = 0; i < 3; ++i) {
    if (!isfinite(W.host[i])) throw Error(OT_ERR_NONFINITE, "non-finite residual");
    if (norms) norms[i] = sqrt(W.host[i]);
    t += W.host[i];
  }
  return sqrt(t);
}

// Recover the full direction from the projected solution in W.sol (reading R10):
// drho <- P^T drho, dphi <- dphi_hat + per-slice constants, zero mean.
void recover_direction(Workspace& W, Stream st) {
  const Dims& d = W.d;
  double* dphi = W.sol;
  double* drho = W.sol + W.Np;
  double* sm = W.scal + 64;
  k_slice_sums(drho, d.K, d.Nc, 1.0 / (double)d.Nc, sm, st);
  k_slice_shift(drho, d.K, d.Nc, sm, 1.0, st);
  k_kkt_apply(d, W.kcoef, W.sol, W.ytmp, W.xmean, W.wsum, st);
  k_shift_constants(d, W.gsum, W.wsum, 1.0, W.cshift, st);
  k_slice_shift(dphi, d.K + 1, d.N, W.cshift, -1.0, st);
  k_slice_sums(dphi, 1, W.Np, 1.0 / (double)W.Np, sm, st);
  k_slice_shift(dphi, 1, W.Np, sm, 1.0, st);
}

double newton_direction(Workspace& W, const ot_options& opt, double normF, double eps, Stream st) {
  const Dims& d = W.d;
  k_newton_rhs(d, W.Fphi, W.Frho, W.Fs, W.rho, W.rhs, W.hvec, W.gsum, st);
  refresh_coefficients(W, st);
  (void)normF;  // ||F||^2 by components is in W.scal[0..2] (residual_norm)
  fgmres(W, opt, W.rhs, W.sol, eps, W.scal, 3, st);
  recover_direction(W, st);
  k_step_length(d, W.rho, W.s, W.sol + W.Np, W.hvec, W.ds, opt.tau, W.scal + 8, W.partial, st);
  dev::copy_d2h(W.host, W.scal + 8, sizeof(double), st);
  dev::sync(st);
  return W.host[0];
}

// ------------------------------------------------------------------ interior point
int ipm_run(Workspace& W, const ot_options& opt, double mu0, double tol, ot_stats* stats, Stream st) {
  dev::PdlScope pdl_scope(opt.pdl != 0);
  const Dims& d = W.d;
  const int K = d.K;
  const double area_total = 1.0;
  int n_stage = 1;
  {
    double mu = mu0;
    while (mu * area_total * K / (K + 1.0) > tol && n_stage < OT_MAX_STAGES) {
      mu *= opt.mu_factor;
      ++n_stage;
    }
  }
  k_slice_sums(W.r0, 1, d.Nc, d.area_c, W.scal + 16, st);
  dev::copy_d2h(W.host, W.scal + 16, sizeof(double), st);
  dev::sync(st);
  const double mass0 = W.host[0];

  double t_start = dev::now();
  double mu = mu0;
  double f = 0.0;
  int total_newton = 0;
  W.outer_iters = W.inner_iters = W.capped_solves = 0;
  for (int stage = 0; stage < n_stage; ++stage) {
    double t0 = dev::now();
    long long o0 = W.outer_iters, i0 = W.inner_iters;
    double norms[3];
    W.mu = mu;
    f = residual_norm(W, mu, st, norms);
    bool last = stage == n_stage - 1;
    double tolN = ((last && opt.final_newton_tol > 0) ? opt.final_newton_tol : opt.newton_tol) * std::max(1.0, f);
    double eps = (last && opt.final_eps_out > 0) ? opt.final_eps_out : opt.eps_out;
    int steps = 0;
    while (f > tolN) {
      if (steps >= opt.max_newton) {
        char buf[160];
        snprintf(buf, sizeof(buf), "Newton did not converge at mu=%g: ||F||=%.3e after %d steps", mu, f, steps);
        throw Error(OT_ERR_NOT_CONVERGED, buf);
      }
      double alpha = newton_direction(W, opt, f, eps, st);
      if (!(alpha > 0.0) || !isfinite(alpha)) throw Error(OT_ERR_BREAKDOWN, "zero or invalid step length");
      k_update(d, W.scal + 8, 0.0, W.sol, W.sol + W.Np, W.ds, W.phi, W.rho, W.s, st);
      k_slice_sums(W.rho, K, d.Nc, d.area_c, W.mass, st);
      k_rescale(d, W.rho, W.mass, mass0, st);
      f = residual_norm(W, mu, st, norms);
      ++steps;
      if (opt.verbose >= 2)
        fprintf(stderr, "  newton %2d  mu=%.2e  alpha=%.3f  ||F||=%.3e  outer=%lld inner=%lld\n", steps, mu, alpha,
                f, W.outer_iters - o0, W.inner_iters - i0);
    }
    total_newton += steps;
    double t1 = dev::now();
    if (opt.verbose >= 1)
      fprintf(stderr, "stage %2d mu=%.2e newton=%d outer/ls=%.1f inner/outer=%.2f ||F||=%.3e %.3fs\n", stage, mu,
              steps, steps ? (double)(W.outer_iters - o0) / steps : 0.0,
              (W.outer_iters - o0) ? (double)(W.inner_iters - i0) / (double)(W.outer_iters - o0) : 0.0, f, t1 - t0);
    if (stats && stage < OT_MAX_STAGES) {
      stats->stage_mu[stage] = mu;
      stats->stage_newton[stage] = steps;
      stats->stage_outer[stage] = W.outer_iters - o0;
      stats->stage_inner[stage] = W.inner_iters - i0;
      stats->stage_seconds[stage] = t1 - t0;
      stats->stage_residual[stage] = f;
    }
    if (!last) mu *= opt.mu_factor;
  }
  if (stats) {
    stats->stages = n_stage;
    stats->newton_steps = total_newton;
    stats->fgmres_iters = W.outer_iters;
    stats->inner_iters = W.inner_iters;
    stats->final_residual = f;
    stats->mu = mu;
    stats->gap = mu * area_total * K / (K + 1.0);
    stats->seconds = dev::now() - t_start;
  }
  return total_newton;
}

}  // namespace ot
