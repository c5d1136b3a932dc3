// mg_body.cuh -- per-cell bodies of the multigrid smoothers and level operator.
//
// Level operator for slice k, cell c (alpha [slot][slice][cell], tau [slice][cell]):
//   (M x)^k_c = sum_slot alpha^k_{c,slot} (x^k_c - x^k_o) + tau^k_c (2 x^k_c - x^{k-1}_c - x^{k+1}_c),
// x^{-1} = x^S = 0; tau absent for the time-slice Laplacians.
#pragma once
#include "ot_internal.h"

namespace ot {

// Quotients of the FP32 smoothers use the fast hardware division (about 2 ulp;
// a smoother needs no correctly rounded quotient); FP64 divides exactly.
OT_HD float mg_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
OT_HD double mg_div(double a, double b) { return a / b; }

// Point update of cell c in slice k: x = (b + sum alpha x_o) / sum alpha.
template <typename T>
OT_HD void point_gs(int S, const LevelView<T>& L, int k, i64 c) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  const T* xs = L.x + (i64)k * L.ld;
  T num = L.b[(i64)k * L.ld + c], den = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    T a = L.alpha[((i64)sl * S + k) * L.ld + c];
    den += a;
    if (nb[sl] >= 0) num += a * xs[nb[sl]];
  }
  L.x[(i64)k * L.ld + c] = mg_div(num, den);
}

// Line update of cell c: solve the time-tridiagonal system with the spatial neighbours frozen.
template <typename T>
OT_HD void line_gs(int S, const LevelView<T>& L, i64 c, T* lc, T* lr) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  i64 nc = L.ld;  // slice stride
  T cp = 0, rp = 0;
  for (int k = 0; k < S; ++k) {
    const T* xs = L.x + (i64)k * nc;
    T dg = 2 * L.tau[(i64)k * nc + c], rhs = L.b[(i64)k * nc + c];
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      T a = L.alpha[((i64)sl * S + k) * nc + c];
      dg += a;
      if (nb[sl] >= 0) rhs += a * xs[nb[sl]];
    }
    T off = -L.tau[(i64)k * nc + c];  // coefficient of x^{k-1} and of x^{k+1}
    T sub = (k > 0) ? off : (T)0;
    T den = dg - sub * cp;
    cp = (k < S - 1) ? off / den : (T)0;
    rp = (rhs - sub * rp) / den;
    lc[(i64)k * nc + c] = cp;
    lr[(i64)k * nc + c] = rp;
  }
  T xn = 0;
  for (int k = S - 1; k >= 0; --k) {
    T v = lr[(i64)k * nc + c] - lc[(i64)k * nc + c] * xn;
    L.x[(i64)k * nc + c] = v;
    xn = v;
  }
}

template <typename T>
OT_HD T level_apply(int S, const LevelView<T>& L, int k, i64 c) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  const T* xs = L.x + (i64)k * L.ld;
  T xc = xs[c], acc = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    acc += L.alpha[((i64)sl * S + k) * L.ld + c] * (xc - xs[nb[sl]]);
  }
  if (L.tau) {
    T xm = (k > 0) ? L.x[(i64)(k - 1) * L.ld + c] : (T)0;
    T xp = (k < S - 1) ? L.x[(i64)(k + 1) * L.ld + c] : (T)0;
    acc += L.tau[(i64)k * L.ld + c] * (2 * xc - xm - xp);
  }
  return acc;
}

// Space-time level of side 1 (two triangles per slice, coupled through their
// shared diagonal edge, slot 0): the block-tridiagonal system with 2x2
// blocks along time, solved exactly by one thread (block Thomas).  Row (k, c):
// (sum_slot alpha) x_c - alpha_0 x_other + tau (2 x_c - x_c^{k-1} - x_c^{k+1}) = b.
// G: scratch of 4 S; the forward right-hand sides go to r.
template <typename T>
OT_HD void coarse_exact_side1(int S, const LevelView<T>& L, T* G) {
  const i64 ld = L.ld;
  T p00 = 0, p01 = 0, p10 = 0, p11 = 0, q0 = 0, q1 = 0;  // G_{k-1}, g_{k-1}
  for (int k = 0; k < S; ++k) {
    const i64 o = (i64)k * ld;
    const T t0 = L.tau[o], t1 = L.tau[o + 1];
    T s0 = 2 * t0, s1 = 2 * t1;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      s0 += L.alpha[((i64)sl * S + k) * ld];
      s1 += L.alpha[((i64)sl * S + k) * ld + 1];
    }
    const T e0 = L.alpha[o], e1 = L.alpha[o + 1];  // slot 0, slice k
    // A_k = D_k - L_k G_{k-1} with L_k = diag(-t0, -t1)
    const T a00 = s0 + t0 * p00, a01 = -e0 + t0 * p01, a10 = -e1 + t1 * p10, a11 = s1 + t1 * p11;
    const T b0 = L.b[o] + t0 * q0, b1 = L.b[o + 1] + t1 * q1;
    const T id = (T)1 / (a00 * a11 - a01 * a10);
    q0 = id * (a11 * b0 - a01 * b1);
    q1 = id * (a00 * b1 - a10 * b0);
    // G_k = A_k^{-1} U_k with U_k = diag(-t0, -t1) (zero in the last slice)
    const T u0 = (k < S - 1) ? -t0 : (T)0, u1 = (k < S - 1) ? -t1 : (T)0;
    p00 = id * a11 * u0;
    p01 = -id * a01 * u1;
    p10 = -id * a10 * u0;
    p11 = id * a00 * u1;
    G[4 * k] = p00;
    G[4 * k + 1] = p01;
    G[4 * k + 2] = p10;
    G[4 * k + 3] = p11;
    L.r[o] = q0;
    L.r[o + 1] = q1;
  }
  T x0 = 0, x1 = 0;
  for (int k = S - 1; k >= 0; --k) {
    const i64 o = (i64)k * ld;
    const T y0 = L.r[o] - (G[4 * k] * x0 + G[4 * k + 1] * x1);
    const T y1 = L.r[o + 1] - (G[4 * k + 2] * x0 + G[4 * k + 3] * x1);
    L.x[o] = y0;
    L.x[o + 1] = y1;
    x0 = y0;
    x1 = y1;
  }
}

}  // namespace ot
