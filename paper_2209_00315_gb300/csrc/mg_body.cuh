// mg_body.cuh -- per-cell bodies of the multigrid smoothers and level operator.
//
// Level operator for slice k, cell c (alpha [slot][slice][cell], tau [slice][cell]):
//   (M x)^k_c = sum_slot alpha^k_{c,slot} (x^k_c - x^k_o) + tau^k_c (2 x^k_c - x^{k-1}_c - x^{k+1}_c),
// x^{-1} = x^S = 0; tau absent for the time-slice Laplacians.
#pragma once
#include "ot_internal.h"

namespace ot {

// Point update of cell c in slice k: x = (b + sum alpha x_o) / sum alpha.
template <typename T>
OT_HD void point_gs(int S, const LevelView<T>& L, int k, i64 c) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  const T* xs = L.x + (i64)k * L.nc;
  T num = L.b[(i64)k * L.nc + c], den = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    T a = L.alpha[((i64)sl * S + k) * L.nc + c];
    den += a;
    if (nb[sl] >= 0) num += a * xs[nb[sl]];
  }
  L.x[(i64)k * L.nc + c] = num / den;
}

// Line update of cell c: solve the time-tridiagonal system with the spatial neighbours frozen.
template <typename T>
OT_HD void line_gs(int S, const LevelView<T>& L, i64 c, T* lc, T* lr) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  i64 nc = L.nc;
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
  const T* xs = L.x + (i64)k * L.nc;
  T xc = xs[c], acc = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    acc += L.alpha[((i64)sl * S + k) * L.nc + c] * (xc - xs[nb[sl]]);
  }
  if (L.tau) {
    T xm = (k > 0) ? L.x[(i64)(k - 1) * L.nc + c] : (T)0;
    T xp = (k < S - 1) ? L.x[(i64)(k + 1) * L.nc + c] : (T)0;
    acc += L.tau[(i64)k * L.nc + c] * (2 * xc - xm - xp);
  }
  return acc;
}

}  // namespace ot
