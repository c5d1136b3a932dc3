// stencil.cuh -- per-element bodies of every stencil of the path.
//
// Each function computes one output entry from plain pointers; the CUDA
// kernels call them once per thread.  All geometry is arithmetic on the
// structured right-triangle grids:
//
//   grid of side m: squares (I, J), 0 <= I, J < m, side h = 1/m; square (I, J)
//   holds the lower-right triangle L = (t=0) and the upper-left U = (t=1),
//   cell index t m^2 + J m + I, area h^2/2.
//   Interior edges and their two-point transmissibility |e|/|w|:
//     diagonal of (I,J): L(I,J) | U(I,J)      |e| = sqrt2 h, |w| = sqrt2 h/3 -> 3
//     right of (I,J):    L(I,J) | U(I+1,J)    |e| = h, |w| = h            -> 1
//     top of (I,J):      U(I,J) | L(I,J+1)    |e| = h, |w| = h            -> 1
//   (|w| on the diagonals is the barycentre distance: the circumcentres of the
//   two right triangles coincide there.)  Every cell has three edge slots:
//     L: 0 -> U(I,J), 1 -> U(I+1,J), 2 -> U(I,J-1)
//     U: 0 -> L(I,J), 1 -> L(I-1,J), 2 -> L(I,J+1)
//   and the mesh graph is bipartite: every neighbour of an L cell is a U cell.
//
//   Two levels (Sec. 2.1): the fine grid (side 2n, potential) is the midpoint
//   4-split of the coarse grid (side n, density).  Fine square (I, J) lies in
//   coarse square (I/2, J/2); of its two triangles, only the upper-left one of
//   sub-square (0,1) and the lower-right one of sub-square (1,0) belong to the
//   other coarse triangle than their type says.
//
//   All edge reconstructions use weight 1/2 on each side (lambda_e = 1/2 on this
//   mesh), so R_E rho on a fine edge is the mean of the two parents' values and
//   W_e (grad u)_e (grad v)_e = T_e (u_c - u_o)(v_c - v_o) for |e||w| = W_e.
#pragma once
#include <stdint.h>

#ifndef OT_HD
#ifdef __CUDACC__
#define OT_HD __host__ __device__ __forceinline__
#else
#define OT_HD inline
#endif
#endif

namespace ot {

typedef long long i64;

// Sizes of one problem: coarse side n, fine side m = 2n, K density slices.
struct Dims {
  int n, m, K;
  i64 N, Nc;            // fine / coarse cells per slice
  double dt;            // 1/(K+1)
  double area_f, area_c;
  double af_dt;         // area_f / dt
};

OT_HD Dims make_dims(int n, int K) {
  Dims d;
  d.n = n;
  d.m = 2 * n;
  d.K = K;
  d.Nc = 2LL * n * n;
  d.N = 2LL * d.m * d.m;
  d.dt = 1.0 / (K + 1);
  d.area_c = 0.5 / ((double)n * n);
  d.area_f = 0.5 / ((double)d.m * d.m);
  d.af_dt = d.area_f / d.dt;
  return d;
}

OT_HD double trans(int slot) { return slot == 0 ? 3.0 : 1.0; }

struct Cell {
  int t, I, J;
};

// In-slice indices stay below 2 m^2 <= 2^25, so 32-bit arithmetic is exact and
// keeps 64-bit integer division out of every stencil.
OT_HD Cell decode(int m, i64 c) {
  Cell q;
  int cc = (int)c, mm = m * m;
  q.t = cc >= mm ? 1 : 0;
  int r = cc - q.t * mm;
  q.J = r / m;
  q.I = r - q.J * m;
  return q;
}

OT_HD i64 encode(int m, int t, int I, int J) { return (i64)(t * m * m + J * m + I); }

// Neighbour of each edge slot, -1 on the domain boundary (no-flux edges are dropped).
OT_HD void neighbours(int m, const Cell& q, i64 nb[3]) {
  if (q.t == 0) {
    nb[0] = encode(m, 1, q.I, q.J);
    nb[1] = (q.I + 1 < m) ? encode(m, 1, q.I + 1, q.J) : -1;
    nb[2] = (q.J > 0) ? encode(m, 1, q.I, q.J - 1) : -1;
  } else {
    nb[0] = encode(m, 0, q.I, q.J);
    nb[1] = (q.I > 0) ? encode(m, 0, q.I - 1, q.J) : -1;
    nb[2] = (q.J + 1 < m) ? encode(m, 0, q.I, q.J + 1) : -1;
  }
}

// The same, also returning the neighbours' (t, I, J) (valid where nb >= 0).
OT_HD void neighbours(int m, const Cell& q, i64 nb[3], Cell nq[3]) {
  int to = 1 - q.t;
  nq[0] = Cell{to, q.I, q.J};
  if (q.t == 0) {
    nq[1] = Cell{to, q.I + 1, q.J};
    nq[2] = Cell{to, q.I, q.J - 1};
  } else {
    nq[1] = Cell{to, q.I - 1, q.J};
    nq[2] = Cell{to, q.I, q.J + 1};
  }
  nb[0] = encode(m, nq[0].t, nq[0].I, nq[0].J);
  nb[1] = (nq[1].I >= 0 && nq[1].I < m) ? encode(m, nq[1].t, nq[1].I, nq[1].J) : -1;
  nb[2] = (nq[2].J >= 0 && nq[2].J < m) ? encode(m, nq[2].t, nq[2].I, nq[2].J) : -1;
}

// Coarse triangle (grid side m/2) containing fine cell q (grid side m): the injection J.
OT_HD i64 parent(int m, const Cell& q) {
  int n = m >> 1;
  int a = q.I & 1, b = q.J & 1;
  int tc = (q.t == 0) ? ((a == 0 && b == 1) ? 1 : 0) : ((a == 1 && b == 0) ? 0 : 1);
  return encode(n, tc, q.I >> 1, q.J >> 1);
}

OT_HD i64 parent_of(int m, i64 c) { return parent(m, decode(m, c)); }

// The four fine cells (grid side 2n) of coarse cell q (grid side n).
OT_HD void children(int n, const Cell& q, i64 ch[4]) {
  int m = 2 * n, I = 2 * q.I, J = 2 * q.J;
  if (q.t == 0) {
    ch[0] = encode(m, 0, I, J);
    ch[1] = encode(m, 0, I + 1, J + 1);
    ch[2] = encode(m, 0, I + 1, J);
    ch[3] = encode(m, 1, I + 1, J);
  } else {
    ch[0] = encode(m, 1, I, J);
    ch[1] = encode(m, 1, I + 1, J + 1);
    ch[2] = encode(m, 0, I, J + 1);
    ch[3] = encode(m, 1, I, J + 1);
  }
}

// rho^k for k = 0..K+1 (paper index): boundary data at k = 0 and k = K+1.
template <typename T>
OT_HD T rho_at(const Dims& d, const T* rho, const T* r0, const T* r1, int k, i64 C) {
  return k == 0 ? r0[C] : (k == d.K + 1 ? r1[C] : rho[(i64)(k - 1) * d.Nc + C]);
}

// Mean density of phi slice jj (paper j = jj+1) on coarse cell C: (rho^{j-1} + rho^j)/2.
template <typename T>
OT_HD T rho_bar(const Dims& d, const T* rho, const T* r0, const T* r1, int jj, i64 C) {
  return (T)0.5 * (rho_at(d, rho, r0, r1, jj, C) + rho_at(d, rho, r0, r1, jj + 1, C));
}

// ----------------------------------------------------------------- residual
// F_phi^j on fine cell c, phi slice jj = j-1 (Eq. conservation_discrete):
//   -|c| (rho^j - rho^{j-1})_P/dt + sum_e T_e rho~^j_e (phi_c - phi_o).
OT_HD double residual_phi(const Dims& d, const double* phi, const double* rho, const double* r0,
                          const double* r1, int jj, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  i64 P = parent(d.m, q);
  const double* ph = phi + (i64)jj * d.N;
  double ra = rho_at(d, rho, r0, r1, jj, P), rb = rho_at(d, rho, r0, r1, jj + 1, P);
  double rc = 0.5 * (ra + rb);
  double acc = -d.area_f * (rb - ra) / d.dt;
  double pc = ph[c];
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    double ro = rho_bar(d, rho, r0, r1, jj, parent(d.m, nq[sl]));
    acc += trans(sl) * 0.5 * (rc + ro) * (pc - ph[nb[sl]]);
  }
  return acc;
}

// F_rho^k on coarse cell C, rho slice k0 = k-1 (Eq. hj_discrete, time term J^T M):
//   sum_{c in C} [ |c| (phi^{k+1} - phi^k)_c/dt + 1/8 sum_e T_e ((dphi^k_e)^2 + (dphi^{k+1}_e)^2) ] + |c'| s^k_C.
// (R_T q = 1/2 sum_{c in C} sum_{e at c} W_e q_e counts interior fine edges twice at 1/2.)
OT_HD double residual_rho(const Dims& d, const double* phi, const double* s, int k0, i64 C) {
  Cell qc = decode(d.n, C);
  i64 ch[4];
  children(d.n, qc, ch);
  const double* p0 = phi + (i64)k0 * d.N;
  const double* p1 = p0 + d.N;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    i64 c = ch[a];
    Cell q = decode(d.m, c);
    i64 nb[3];
    Cell nq[3];
    neighbours(d.m, q, nb, nq);
    acc += d.area_f * (p1[c] - p0[c]) / d.dt;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      if (nb[sl] < 0) continue;
      double g0 = p0[c] - p0[nb[sl]], g1 = p1[c] - p1[nb[sl]];
      acc += 0.125 * trans(sl) * (g0 * g0 + g1 * g1);
    }
  }
  return acc + d.area_c * s[(i64)k0 * d.Nc + C];
}

// ----------------------------------------------------------------- KKT operator
// phi rows of [A, B^T P^T] x, phi slice jj (paper j = jj+1), with y = P^T x_rho (slice means xmean removed):
//   sum_e T_e [rho~^j_e (x_c - x_o) + (ybar^j_Pc + ybar^j_Po)/2 (phi_c - phi_o)] + |c| (y^{j-1} - y^j)_Pc/dt,
//   ybar^j = (y^{j-1} + y^j)/2, y^0 = y^{K+1} = 0.  with_a = false drops the A term.
template <typename T>
OT_HD T kkt_phi(const Dims& d, const T* phi, const T* rho, const T* r0, const T* r1,
                     const T* xp, const T* xr, const T* xmean, bool with_a, int jj, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  i64 P = parent(d.m, q);
  const T* ph = phi + (i64)jj * d.N;
  const T* xs = xp + (i64)jj * d.N;
  const T* ym = (jj >= 1) ? xr + (i64)(jj - 1) * d.Nc : nullptr;
  const T* yp = (jj <= d.K - 1) ? xr + (i64)jj * d.Nc : nullptr;
  T mm = (jj >= 1) ? xmean[jj - 1] : (T)0, mp = (jj <= d.K - 1) ? xmean[jj] : (T)0;
  T yma = ym ? ym[P] - mm : (T)0, ypa = yp ? yp[P] - mp : (T)0;
  T acc = (T)d.area_f * (yma - ypa) / (T)d.dt;
  T ybc = (T)0.5 * (yma + ypa);
  T rc = with_a ? rho_bar(d, rho, r0, r1, jj, P) : (T)0;
  T pc = ph[c], xc = with_a ? xs[c] : (T)0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    i64 o = nb[sl];
    i64 Po = parent(d.m, nq[sl]);
    T ybo = (T)0.5 * ((ym ? ym[Po] - mm : (T)0) + (yp ? yp[Po] - mp : (T)0));
    T term = (T)0.5 * (ybc + ybo) * (pc - ph[o]);
    if (with_a) term += (T)0.5 * (rc + rho_bar(d, rho, r0, r1, jj, Po)) * (xc - xs[o]);
    acc += (T)trans(sl) * term;
  }
  return acc;
}

// (B x)^k on coarse cell C, rho slice k0 = k-1 (Sec. 3, B = J^T D_t M + H G D_x):
//   sum_{c in C} [ |c| (x^{k+1} - x^k)_c/dt
//                  + 1/4 sum_e T_e ((phi^k_c - phi^k_o)(x^k_c - x^k_o) + (same at k+1)) ].
template <typename T>
OT_HD T apply_B(const Dims& d, const T* phi, const T* x, int k0, i64 C) {
  Cell qc = decode(d.n, C);
  i64 ch[4];
  children(d.n, qc, ch);
  const T* p0 = phi + (i64)k0 * d.N;
  const T* p1 = p0 + d.N;
  const T* x0 = x + (i64)k0 * d.N;
  const T* x1 = x0 + d.N;
  T acc = (T)0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    i64 c = ch[a];
    Cell q = decode(d.m, c);
    i64 nb[3];
    Cell nq[3];
    neighbours(d.m, q, nb, nq);
    acc += (T)d.area_f * (x1[c] - x0[c]) / (T)d.dt;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      if (nb[sl] < 0) continue;
      i64 o = nb[sl];
      acc += (T)0.25 * (T)trans(sl) * ((p0[c] - p0[o]) * (x0[c] - x0[o]) + (p1[c] - p1[o]) * (x1[c] - x1[o]));
    }
  }
  return acc;
}

// rho rows before projection: w = B x_phi - C P^T x_rho, C = M' diag(s/rho).
template <typename T>
OT_HD T kkt_rho(const Dims& d, const T* phi, const T* rho, const T* s, const T* xp,
                     const T* xr, const T* xmean, int k0, i64 C) {
  i64 idx = (i64)k0 * d.Nc + C;
  T xh = xr[idx] - xmean[k0];
  return apply_B(d, phi, xp, k0, C) - (T)d.area_c * s[idx] / rho[idx] * xh;
}

// ----------------------------------------------------------------- KKT with edge coefficients
// The KKT rows above spend most of their time on FP64 arithmetic that depends
// only on (phi, rho): the edge weights of the A block and the potential
// differences of the B block.  Computed once per Newton step into
//   kc[(jj*6 + sl)*N + c]     = w = T_e (rho~_c + rho~_o)/2,
//   kc[(jj*6 + 3 + sl)*N + c] = g = T_e (phi^jj_c - phi^jj_o)/2   (zero on boundary slots),
//   kc[(K+1)*6*N + k0*N' + C] = |C| s/rho,
// every later operator application is loads plus a few FMAs per row.  The
// 2(K+1)N' values after those are scratch of each application (the slice
// values of kkt_slice_values).
OT_HD i64 kkt_yb_offset(const Dims& d) { return (i64)(d.K + 1) * 6 * d.N + (i64)d.K * d.Nc; }
// After the slice values: per potential slice and fine cell, the edge sum
// e^jj_c = sum_slot g_slot (x^jj_c - x^jj_o) of the B part, written by the phi
// rows of an application and summed over the four children by its rho rows.
OT_HD i64 kkt_e_offset(const Dims& d) { return kkt_yb_offset(d) + 2LL * (d.K + 1) * d.Nc; }
OT_HD i64 kkt_coef_count(const Dims& d) { return kkt_e_offset(d) + (i64)(d.K + 1) * d.N; }

OT_HD void kkt_edge_coef(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                         int jj, i64 c, double w[3], double g[3]) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  const double* ph = phi + (i64)jj * d.N;
  const double rc = rho_bar(d, rho, r0, r1, jj, parent(d.m, q));
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) {
      w[sl] = 0.0;
      g[sl] = 0.0;
      continue;
    }
    const double t = trans(sl);
    w[sl] = t * (0.5 * (rc + rho_bar(d, rho, r0, r1, jj, parent(d.m, nq[sl]))));
    g[sl] = t * (0.5 * (ph[c] - ph[nb[sl]]));
  }
}

// The B^T P^T part of the phi rows depends on x_rho only through, per
// potential slice jj and coarse cell C (y = x_rho minus its slice means,
// y^{-1} = y^{K} = 0 at the ends):
//   ybar^jj_C  = (y^{jj-1}_C + y^jj_C)/2,   ydif^jj_C = |c| (y^{jj-1}_C - y^jj_C)/dt.
// yb holds ybar for jj = 0..K, then ydif.
OT_HD void kkt_slice_values(const Dims& d, const double* xr, const double* xmean, int jj, i64 C, double* yb) {
  const double ym = (jj >= 1) ? xr[(i64)(jj - 1) * d.Nc + C] - xmean[jj - 1] : 0.0;
  const double yp = (jj <= d.K - 1) ? xr[(i64)jj * d.Nc + C] - xmean[jj] : 0.0;
  yb[(i64)jj * d.Nc + C] = 0.5 * (ym + yp);
  yb[(i64)(d.K + 1 + jj) * d.Nc + C] = d.af_dt * (ym - yp);
}

// kkt_phi from the edge coefficients and the slice values of kkt_slice_values
// (with_a = false: the B^T P^T part only): three FMA pairs per row.
OT_HD double kkt_phi_sliced(const Dims& d, const double* kc, const double* xp, const double* yb, bool with_a,
                            int jj, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  const i64 P = parent(d.m, q);
  const double* ybar = yb + (i64)jj * d.Nc;
  const double* xs = xp + (i64)jj * d.N;
  double acc = yb[(i64)(d.K + 1 + jj) * d.Nc + P];
  const double ybc = ybar[P];
  const double xc = with_a ? xs[c] : 0.0;
  const double* kw = kc + (i64)jj * 6 * d.N + c;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    acc += kw[(i64)(3 + sl) * d.N] * (ybc + ybar[parent(d.m, nq[sl])]);
    if (with_a) acc += kw[(i64)sl * d.N] * (xc - xs[nb[sl]]);
  }
  return acc;
}

// (B x)^k on coarse cell C from the edge coefficients: 1/4 T_e dphi dx = g dx / 2.
OT_HD double apply_B_cached(const Dims& d, const double* kc, const double* x, int k0, i64 C) {
  i64 ch[4];
  children(d.n, decode(d.n, C), ch);
  const double* x0 = x + (i64)k0 * d.N;
  const double* x1 = x0 + d.N;
  const double* g0 = kc + ((i64)k0 * 6 + 3) * d.N;
  const double* g1 = kc + ((i64)(k0 + 1) * 6 + 3) * d.N;
  double dtime = 0.0, edges = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    i64 c = ch[a];
    i64 nb[3];
    neighbours(d.m, decode(d.m, c), nb);
    const double x0c = x0[c], x1c = x1[c];
    dtime += x1c - x0c;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      if (nb[sl] < 0) continue;
      i64 o = nb[sl];
      edges += g0[(i64)sl * d.N + c] * (x0c - x0[o]) + g1[(i64)sl * d.N + c] * (x1c - x1[o]);
    }
  }
  return d.af_dt * dtime + 0.5 * edges;
}

// ----------------------------------------------------------------- BB pieces
// u = M^{-1} B~ z on fine cell c, phi slice jj (paper j = jj+1), reading of Sec. 4.3.2:
//   (z^j - z^{j-1})_Pc/dt + 1/(2|c|) sum_e T_e (phi^j_c - phi^j_o)(zbar^j_Pc - zbar^j_Po),
//   zbar^j = (z^{j-1} + z^j)/2, z^0 = z^{K+1} = 0.
template <typename T>
OT_HD T schur_u(const Dims& d, const T* phi, const T* z, int jj, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  i64 P = parent(d.m, q);
  const T* ph = phi + (i64)jj * d.N;
  const T* zm = (jj >= 1) ? z + (i64)(jj - 1) * d.Nc : nullptr;
  const T* zp = (jj <= d.K - 1) ? z + (i64)jj * d.Nc : nullptr;
  T zmc = zm ? zm[P] : (T)0, zpc = zp ? zp[P] : (T)0;
  T zbc = (T)0.5 * (zmc + zpc);
  T acc = (T)0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    i64 Po = parent(d.m, nq[sl]);
    T zbo = (T)0.5 * ((zm ? zm[Po] : (T)0) + (zp ? zp[Po] : (T)0));
    acc += (T)trans(sl) * (ph[c] - ph[nb[sl]]) * (zbc - zbo);
  }
  return (zpc - zmc) / (T)d.dt + (T)0.5 * acc / (T)d.area_f;
}

// (A~^k z)_C on the coarse grid: sum_E T_E (rho^k_C + rho^k_O)/2 (z_C - z_O).
template <typename T>
OT_HD T apply_atilde(const Dims& d, const T* rho, const T* z, int k0, i64 C) {
  Cell q = decode(d.n, C);
  i64 nb[3];
  neighbours(d.n, q, nb);
  const T* rk = rho + (i64)k0 * d.Nc;
  const T* zk = z + (i64)k0 * d.Nc;
  T acc = (T)0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    acc += (T)trans(sl) * (T)0.5 * (rk[C] + rk[nb[sl]]) * (zk[C] - zk[nb[sl]]);
  }
  return acc;
}

// Schur operator row (Eq. pseudoschur-bis): s (A~ z) - rho (B u) with u = M^{-1} B~ z.
template <typename T>
OT_HD T schur_out(const Dims& d, const T* phi, const T* rho, const T* s, const T* u,
                       const T* z, int k0, i64 C) {
  i64 idx = (i64)k0 * d.Nc + C;
  return s[idx] * apply_atilde(d, rho, z, k0, C) - rho[idx] * apply_B(d, phi, u, k0, C);
}

// ----------------------------------------------------------------- cost, dual
// Contribution of fine cell c, phi slice jj, to sum_e W rho~ (grad phi)^2 / 2: each edge is
// visited from both sides, so the cell adds 1/4 sum_e T_e rho~_e (phi_c - phi_o)^2.
OT_HD double cost_cell(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                       int jj, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  i64 P = parent(d.m, q);
  const double* ph = phi + (i64)jj * d.N;
  double rc = rho_bar(d, rho, r0, r1, jj, P);
  double acc = 0.0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    double g = ph[c] - ph[nb[sl]];
    acc += trans(sl) * 0.5 * (rc + rho_bar(d, rho, r0, r1, jj, parent(d.m, nq[sl]))) * g * g;
  }
  return 0.25 * acc;
}

// Contribution of fine cell c to the dual value D:
//   |c| (phi^{K+1}_c rho_f,Pc - phi^1_c rho_in,Pc)
//   - dt/4 * 1/2 sum_e T_e [R_E rho_in]_e (dphi^1_e)^2 + [R_E rho_f]_e (dphi^{K+1}_e)^2.
OT_HD double dual_cell(const Dims& d, const double* phi, const double* r0, const double* r1, i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  i64 P = parent(d.m, q);
  const double* pa = phi;
  const double* pb = phi + (i64)d.K * d.N;
  double acc = d.area_f * (pb[c] * r1[P] - pa[c] * r0[P]);
  double corr = 0.0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    i64 o = nb[sl], Po = parent(d.m, nq[sl]);
    double ga = pa[c] - pa[o], gb = pb[c] - pb[o];
    corr += trans(sl) * (0.5 * (r0[P] + r0[Po]) * ga * ga + 0.5 * (r1[P] + r1[Po]) * gb * gb);
  }
  return acc - 0.25 * d.dt * 0.5 * corr;
}

// ----------------------------------------------------------------- adjoint
// (A^j x^j)_c = sum_e T_e rho~^j_e (x_c - x_o), phi slice jj.
OT_HD double lap_apply(const Dims& d, const double* rho, const double* r0, const double* r1, const double* x, int jj,
                       i64 c) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  const double* xs = x + (i64)jj * d.N;
  double rc = rho_bar(d, rho, r0, r1, jj, parent(d.m, q));
  double acc = 0.0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    if (nb[sl] < 0) continue;
    acc += trans(sl) * 0.5 * (rc + rho_bar(d, rho, r0, r1, jj, parent(d.m, nq[sl]))) * (xs[c] - xs[nb[sl]]);
  }
  return acc;
}

// 1/4 (R_T (grad phi^a)^2)_C = 1/8 sum_{c in C} sum_e T_e (dphi^a_e)^2 for phi slice ja.
OT_HD double kinetic_rho(const Dims& d, const double* phi, int ja, i64 C) {
  Cell qc = decode(d.n, C);
  i64 ch[4];
  children(d.n, qc, ch);
  const double* p = phi + (i64)ja * d.N;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    i64 c = ch[a];
    i64 nb[3];
    neighbours(d.m, decode(d.m, c), nb);
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      if (nb[sl] < 0) continue;
      double g = p[c] - p[nb[sl]];
      acc += 0.125 * trans(sl) * g * g;
    }
  }
  return acc;
}

// lambda^T dF_phi^{ja+1}/d(boundary density) on coarse cell C, for ja = 0 (rho_in, sign = +1)
// or ja = K (rho_f, sign = -1):
//   sum_{c in C} [ sign |c| lambda_c / dt + 1/4 sum_e T_e (phi_c - phi_o)(lambda_c - lambda_o) ].
OT_HD double adjoint_boundary(const Dims& d, const double* phi, const double* lam, int ja, double sign, i64 C) {
  Cell qc = decode(d.n, C);
  i64 ch[4];
  children(d.n, qc, ch);
  const double* p = phi + (i64)ja * d.N;
  const double* l = lam + (i64)ja * d.N;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    i64 c = ch[a];
    i64 nb[3];
    neighbours(d.m, decode(d.m, c), nb);
    acc += sign * d.area_f * l[c] / d.dt;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      if (nb[sl] < 0) continue;
      acc += 0.25 * trans(sl) * (p[c] - p[nb[sl]]) * (l[c] - l[nb[sl]]);
    }
  }
  return acc;
}

// ----------------------------------------------------------------- multigrid
// Level operators have, per (slice, cell), three row coefficients alpha[slot]
// (spatial couplings alpha (x_c - x_o)) and, for the space-time Schur
// hierarchy, a time coefficient tau coupling the cell to itself at k-1, k+1:
//   (M x)^k_c = sum_slot alpha^k_{c,slot} (x^k_c - x^k_o) + tau^k_c (2 x^k_c - x^{k-1}_c - x^{k+1}_c),
// with x^{-1} = x^K = 0 (Dirichlet in time).  Coefficients are stored
// [slot][slice][cell].

// Coarse coefficient from the fine level (side m -> m/2): the Galerkin sum of
// the two fine edges making up each coarse edge, halved for the spatial
// (second-order) part; tau is summed over the four children.  The two fine
// cells below own, in the same slot, the two fine edges of the coarse edge:
//   coarse L(i,j): slot0 <- L(2i,2j).0, L(2i+1,2j+1).0; slot1 <- L(2i+1,2j).1, L(2i+1,2j+1).1;
//                  slot2 <- L(2i,2j).2, L(2i+1,2j).2
//   coarse U(i,j): slot0 <- U(2i,2j).0, U(2i+1,2j+1).0; slot1 <- U(2i,2j).1, U(2i,2j+1).1;
//                  slot2 <- U(2i,2j+1).2, U(2i+1,2j+1).2
OT_HD void coarse_coef_sources(int mc, i64 C, int sl, i64 src[2]) {
  Cell q = decode(mc, C);
  int m = 2 * mc, I = 2 * q.I, J = 2 * q.J;
  if (q.t == 0) {
    if (sl == 0) { src[0] = encode(m, 0, I, J); src[1] = encode(m, 0, I + 1, J + 1); }
    else if (sl == 1) { src[0] = encode(m, 0, I + 1, J); src[1] = encode(m, 0, I + 1, J + 1); }
    else { src[0] = encode(m, 0, I, J); src[1] = encode(m, 0, I + 1, J); }
  } else {
    if (sl == 0) { src[0] = encode(m, 1, I, J); src[1] = encode(m, 1, I + 1, J + 1); }
    else if (sl == 1) { src[0] = encode(m, 1, I, J); src[1] = encode(m, 1, I, J + 1); }
    else { src[0] = encode(m, 1, I, J + 1); src[1] = encode(m, 1, I + 1, J + 1); }
  }
}

// Level-0 coefficients of the slice Laplacian A^j: T_e rho~^j_e.
OT_HD double lap_coef(const Dims& d, const double* rho, const double* r0, const double* r1, int jj, i64 c,
                      int sl) {
  Cell q = decode(d.m, c);
  i64 nb[3];
  Cell nq[3];
  neighbours(d.m, q, nb, nq);
  if (nb[sl] < 0) return 0.0;
  double rc = rho_bar(d, rho, r0, r1, jj, parent(d.m, q));
  double ro = rho_bar(d, rho, r0, r1, jj, parent(d.m, nq[sl]));
  return trans(sl) * 0.5 * (rc + ro);
}

// Level-0 coefficients of the simplified Schur operator on the coarse grid:
//   alpha = s^k_C T_E (rho^k_C + rho^k_O)/2       (the Diag(s) A~ part)
//         + rho^k_C T_E (grad phi . n_E)^2         (two-point form of the spatial part
//                                                   -Diag(rho) B_x M^{-1} B~_x ~ -rho (v.grad)^2),
//   tau   = rho^k_C |c'| / dt^2                    (the time part of -Diag(rho) B M^{-1} B~).
// (grad phi . n_E)^2 is the mean over the two fine edges forming the coarse
// edge and over the potential slices k, k+1 around density time k.
OT_HD double schur_coef(const Dims& d, const double* phi, const double* rho, const double* s, int k0, i64 C,
                        int sl) {
  Cell q = decode(d.n, C);
  i64 nb[3];
  neighbours(d.n, q, nb);
  if (nb[sl] < 0) return 0.0;
  const double* rk = rho + (i64)k0 * d.Nc;
  double coef = s[(i64)k0 * d.Nc + C] * trans(sl) * 0.5 * (rk[C] + rk[nb[sl]]);
  if (phi) {
    // the slot-sl edges of these two fine children make up the coarse edge
    i64 src[2];
    coarse_coef_sources(d.n, C, sl, src);
    double wf = (sl == 0) ? 0.47140452079103168 / d.m : 1.0 / d.m;  // |w| on the fine grid: sqrt2/3 h or h
    double g2 = 0.0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      i64 fnb[3];
      neighbours(d.m, decode(d.m, src[a]), fnb);
      if (fnb[sl] < 0) continue;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const double* p = phi + (i64)(k0 + j) * d.N;
        double g = (p[src[a]] - p[fnb[sl]]) / wf;
        g2 += g * g;
      }
    }
    coef += rk[C] * trans(sl) * 0.25 * g2;
  }
  return coef;
}

OT_HD double schur_tau(const Dims& d, const double* rho, int k0, i64 C) {
  return rho[(i64)k0 * d.Nc + C] * d.area_c / (d.dt * d.dt);
}

// ----------------------------------------------------------------- row layout
// The same geometry for kernels that give a warp one row J of squares and its
// lanes the squares I: a triangle is (t, I, J) and its neighbours and parents
// follow by additions in 32-bit arithmetic, with no index division.  Slot order
// and boundary rule as in neighbours(); parent and children as parent() and
// children().

// Neighbour of slot sl of triangle (t, I, J) on a grid of side m: its index,
// or -1 on the boundary; (I, J) of the neighbour in *Io, *Jo (type 1 - t).
OT_HD int row_nb(int m, int t, int I, int J, int sl, int* Io, int* Jo) {
  int a = I, b = J;
  if (sl == 1) a += (t == 0) ? 1 : -1;
  if (sl == 2) b += (t == 0) ? -1 : 1;
  *Io = a;
  *Jo = b;
  if (a < 0 || a >= m || b < 0 || b >= m) return -1;
  return (1 - t) * m * m + b * m + a;
}

// Coarse triangle (grid side m/2) containing fine triangle (t, I, J) of side m.
OT_HD int row_parent(int m, int t, int I, int J) {
  const int n = m >> 1, a = I & 1, b = J & 1;
  const int tc = (t == 0) ? ((a == 0 && b == 1) ? 1 : 0) : ((a == 1 && b == 0) ? 0 : 1);
  return tc * n * n + (J >> 1) * n + (I >> 1);
}

// The four fine triangles (side 2n) of coarse triangle (t, i, j) of side n, as (type, I, J).
OT_HD void row_children(int t, int i, int j, int ct[4], int cI[4], int cJ[4]) {
  const int I = 2 * i, J = 2 * j;
  if (t == 0) {
    ct[0] = 0, cI[0] = I, cJ[0] = J;
    ct[1] = 0, cI[1] = I + 1, cJ[1] = J + 1;
    ct[2] = 0, cI[2] = I + 1, cJ[2] = J;
    ct[3] = 1, cI[3] = I + 1, cJ[3] = J;
  } else {
    ct[0] = 1, cI[0] = I, cJ[0] = J;
    ct[1] = 1, cI[1] = I + 1, cJ[1] = J + 1;
    ct[2] = 0, cI[2] = I, cJ[2] = J + 1;
    ct[3] = 1, cI[3] = I, cJ[3] = J + 1;
  }
}

}  // namespace ot
