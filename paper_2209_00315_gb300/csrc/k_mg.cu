// k_mg.cu -- geometric multigrid on the nested right-triangle grids.
//
// Two hierarchies share these kernels:
//  * the K+1 time-slice Laplacians A^j (Sec. 3) on the fine grid and its
//    coarsenings: pointwise red-black Gauss-Seidel (L cells, then U cells --
//    the mesh graph is bipartite, so each colour update is exact GS);
//  * the space-time operator that preconditions the BB Schur system
//    (Eq. pseudoschur-bis) on the coarse grid and its coarsenings: the same
//    spatial couplings plus a tridiagonal coupling in time per cell, smoothed
//    by red-black *line* Gauss-Seidel (a Thomas solve along time per cell).
// Transfers are the injection J (prolongation) and its transpose (sum of the
// four children, restriction); coarse operators are the Galerkin sums, halved
// for the second-order spatial part.  Per-thread index arithmetic is in
// stencil.cuh.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "launch.cuh"
#include "mg_body.cuh"

namespace ot {

static inline cudaStream_t cs(Stream s) { return reinterpret_cast<cudaStream_t>(s); }
static constexpr int kT = 256;
static inline int nblk(i64 n) {
  i64 b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : b);
}
#define GRID_LOOP(i, n) for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < (n); i += (i64)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ level-0 coefficients
template <typename T>
__global__ void k_lap_coef0_kernel(Dims d, const double* rho, const double* r0, const double* r1, T* alpha) {
  OT_GRID_DEP_WAIT();
  int S = d.K + 1;
  SLICE_LOOP(jj, S, c, d.N) {
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) alpha[((i64)sl * S + jj) * d.N + c] = (T)lap_coef(d, rho, r0, r1, jj, c, sl);
  }
}

template <typename T>
void k_mg_lap_coef0(const Dims& d, const double* rho, const double* r0, const double* r1, T* alpha, Stream st) {
  launch(k_lap_coef0_kernel<T>, slice_grid(d.N, d.K + 1), kT, 0, cs(st), d, rho, r0, r1, alpha);
}

template <typename T>
__global__ void k_schur_coef0_kernel(Dims d, const double* phi, const double* rho, const double* s, T* alpha,
                                     T* tau) {
  OT_GRID_DEP_WAIT();
  int S = d.K;
  SLICE_LOOP(k0, S, C, d.Nc) {
    i64 i = (i64)k0 * d.Nc + C;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl)
      alpha[((i64)sl * S + k0) * d.Nc + C] = (T)schur_coef(d, phi, rho, s, k0, C, sl);
    tau[i] = (T)schur_tau(d, rho, k0, C);
  }
}

template <typename T>
void k_mg_schur_coef0(const Dims& d, const double* phi, const double* rho, const double* s, T* alpha, T* tau,
                      Stream st) {
  launch(k_schur_coef0_kernel<T>, slice_grid(d.Nc, d.K), kT, 0, cs(st), d, phi, rho, s, alpha, tau);
}

// ------------------------------------------------------------------ coarse coefficients
template <typename T>
__global__ void k_restrict_coef_kernel(int S, LevelView<T> f, LevelView<T> c) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k, S, C, c.nc) {
    i64 i = (i64)k * c.ld + C;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      i64 src[2];
      coarse_coef_sources(c.m, C, sl, src);
      const T* af = f.alpha + ((i64)sl * S + k) * f.ld;
      c.alpha[((i64)sl * S + k) * c.ld + C] = (T)0.5 * (af[src[0]] + af[src[1]]);
    }
    if (c.tau) {
      i64 ch[4];
      children(c.m, decode(c.m, C), ch);
      const T* tf = f.tau + (i64)k * f.ld;
      c.tau[i] = tf[ch[0]] + tf[ch[1]] + tf[ch[2]] + tf[ch[3]];
    }
  }
}

template <typename T>
void k_mg_restrict_coef(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st) {
  launch(k_restrict_coef_kernel<T>, slice_grid(coarse.nc, S), kT, 0, cs(st), S, fine, coarse);
}

// ------------------------------------------------------------------ smoothers
template <typename T>
__global__ void k_point_smooth_kernel(int S, LevelView<T> L, int color) {
  OT_GRID_DEP_WAIT();
  i64 sq = (i64)L.m * L.m;
  SLICE_LOOP(k, S, i, sq) point_gs(S, L, k, (i64)color * sq + i);
}

// Point sweep of one colour in a non-plain mode: neighbour values as
// sweep_neighbour gives them (zero, or x plus the coarse correction).
template <typename T, int MODE>
__global__ void k_point_smooth_mode_kernel(int S, LevelView<T> L, LevelView<T> Lc, int color);

template <typename T>
__global__ void k_line_smooth_kernel(int S, LevelView<T> L, int color, T* lc, T* lr) {
  OT_GRID_DEP_WAIT();
  i64 sq = (i64)L.m * L.m;
  GRID_LOOP(i, sq) line_gs(S, L, (i64)color * sq + i, lc, lr);
}

// ---- warp line solves: parallel cyclic reduction along time.
// A warp owns one cell's time line; lane l holds slices l, l+32, ... (KPL per
// lane, padded with identity equations to 32 KPL), and log2(32 KPL)
// elimination steps replace the K dependent steps of a Thomas sweep.
// Row k: a_k x_{k-s} + d_k x_k + c_k x_{k+s} = r_k at stride s.
template <typename T, int KPL>
__device__ __forceinline__ void pcr_solve(T (&a)[KPL], T (&d)[KPL], T (&c)[KPL], T (&r)[KPL], int lane) {
  constexpr int LOG2 = (KPL == 1) ? 5 : (KPL == 2) ? 6 : 7;
#pragma unroll
  for (int j = 0; j < LOG2; ++j) {
    const int s = 1 << j;
    // each row's 1/d is formed once and travels instead of d: no quotient
    // inside the elimination (a row beyond either end is the identity row)
    T iv[KPL];
#pragma unroll
    for (int q = 0; q < KPL; ++q) iv[q] = mg_div((T)1, d[q]);
    T am[KPL], im[KPL], cm[KPL], rm[KPL], ap[KPL], ip[KPL], cp[KPL], rp[KPL];
    if (s < 32) {
      const int lm = (lane - s) & 31, lp = (lane + s) & 31;
      T xa[KPL], xi[KPL], xc[KPL], xr[KPL], ya[KPL], yi[KPL], yc[KPL], yr[KPL];
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        xa[q] = __shfl_sync(0xffffffffu, a[q], lm);
        xi[q] = __shfl_sync(0xffffffffu, iv[q], lm);
        xc[q] = __shfl_sync(0xffffffffu, c[q], lm);
        xr[q] = __shfl_sync(0xffffffffu, r[q], lm);
        ya[q] = __shfl_sync(0xffffffffu, a[q], lp);
        yi[q] = __shfl_sync(0xffffffffu, iv[q], lp);
        yc[q] = __shfl_sync(0xffffffffu, c[q], lp);
        yr[q] = __shfl_sync(0xffffffffu, r[q], lp);
      }
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        if (lane >= s) {
          am[q] = xa[q]; im[q] = xi[q]; cm[q] = xc[q]; rm[q] = xr[q];
        } else if (q >= 1) {
          am[q] = xa[q - 1]; im[q] = xi[q - 1]; cm[q] = xc[q - 1]; rm[q] = xr[q - 1];
        } else {
          am[q] = 0; im[q] = 1; cm[q] = 0; rm[q] = 0;
        }
        if (lane + s < 32) {
          ap[q] = ya[q]; ip[q] = yi[q]; cp[q] = yc[q]; rp[q] = yr[q];
        } else if (q + 1 < KPL) {
          ap[q] = ya[q + 1]; ip[q] = yi[q + 1]; cp[q] = yc[q + 1]; rp[q] = yr[q + 1];
        } else {
          ap[q] = 0; ip[q] = 1; cp[q] = 0; rp[q] = 0;
        }
      }
    } else {
      const int t = s >> 5;
#pragma unroll
      for (int q = 0; q < KPL; ++q) {
        if (q - t >= 0) {
          am[q] = a[q - t]; im[q] = iv[q - t]; cm[q] = c[q - t]; rm[q] = r[q - t];
        } else {
          am[q] = 0; im[q] = 1; cm[q] = 0; rm[q] = 0;
        }
        if (q + t < KPL) {
          ap[q] = a[q + t]; ip[q] = iv[q + t]; cp[q] = c[q + t]; rp[q] = r[q + t];
        } else {
          ap[q] = 0; ip[q] = 1; cp[q] = 0; rp[q] = 0;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      T al = -a[q] * im[q], ga = -c[q] * ip[q];
      T nd = d[q] + al * cm[q] + ga * ap[q];
      T nr = r[q] + al * rm[q] + ga * rp[q];
      a[q] = al * am[q];
      c[q] = ga * cp[q];
      d[q] = nd;
      r[q] = nr;
    }
  }
}

// Solve of one time line held by a warp, lane l holding rows l KPL .. l KPL + KPL - 1
// as the coefficients of the two substitutions with stored Thomas factors:
//   forward  rp_k = A_k rp_{k-1} + B_k   (A_k = tau_k/den_k, B_k = r_k/den_k, A_0 = 0)
//   back     x_k  = C_k x_{k+1} + rp_k   (C_k = -cp_k, C_{S-1} = 0)
// Both linear recurrences are solved by composing the affine maps within a lane
// and across the warp by a shuffle scan (log2 32 steps).  Rows beyond the line
// carry A = B = C = 0.  On return B holds x.
template <typename T, int KPL>
__device__ __forceinline__ void scan_tridiag(T (&A)[KPL], T (&B)[KPL], const T (&C)[KPL], int lane) {
  T Aa = A[0], Ba = B[0];
#pragma unroll
  for (int q = 1; q < KPL; ++q) {
    Ba = A[q] * Ba + B[q];
    Aa = A[q] * Aa;
  }
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const T Ap = __shfl_up_sync(0xffffffffu, Aa, s), Bp = __shfl_up_sync(0xffffffffu, Ba, s);
    if (lane >= s) {
      Ba = Aa * Bp + Ba;
      Aa = Aa * Ap;
    }
  }
  T rp = __shfl_up_sync(0xffffffffu, Ba, 1);  // rp at the last row of the previous lane
  if (lane == 0) rp = 0;
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    rp = A[q] * rp + B[q];
    B[q] = rp;
  }
  T Cc = C[KPL - 1], Dc = B[KPL - 1];
#pragma unroll
  for (int q = KPL - 2; q >= 0; --q) {
    Dc = C[q] * Dc + B[q];
    Cc = C[q] * Cc;
  }
#pragma unroll
  for (int s = 1; s < 32; s <<= 1) {
    const T Cn = __shfl_down_sync(0xffffffffu, Cc, s), Dn = __shfl_down_sync(0xffffffffu, Dc, s);
    if (lane + s < 32) {
      Dc = Cc * Dn + Dc;
      Cc = Cc * Cn;
    }
  }
  T xn = __shfl_down_sync(0xffffffffu, Dc, 1);  // x at the first row of the next lane
  if (lane == 31) xn = 0;
#pragma unroll
  for (int q = KPL - 1; q >= 0; --q) {
    xn = C[q] * xn + B[q];
    B[q] = xn;
  }
}

// Sweep modes of the smoothers (see k_mg_smooth_mode).
enum { kSweepPlain = 0, kSweepFromZero = 1, kSweepAfterProlong = 2 };

// Value of the spatial neighbour o of slice k as the sweep sees it.
template <typename T, int MODE>
__device__ __forceinline__ T sweep_neighbour(const LevelView<T>& L, const LevelView<T>& Lc, int k, int o) {
  if (MODE == kSweepFromZero) return (T)0;
  T v = L.x[(i64)k * L.ld + o];
  if (MODE == kSweepAfterProlong) v += Lc.x[(i64)k * Lc.ld + parent_of(L.m, o)];
  return v;
}

// The same on a staged level with tables (32-bit indices): the parent of the
// neighbour from the table.
template <typename T, int MODE>
__device__ __forceinline__ T sweep_neighbour_t(const LevelView<T>& L, const LevelView<T>& Lc, int k, int o) {
  if (MODE == kSweepFromZero) return (T)0;
  T v = L.x[k * (int)L.ld + o];
  if (MODE == kSweepAfterProlong) v += Lc.x[k * (int)Lc.ld + L.par[o]];
  return v;
}

// level_apply on a staged level with tables.
template <typename T>
__device__ __forceinline__ T level_apply_t(int S, const LevelView<T>& L, int k, int c) {
  const int ld = (int)L.ld, nc = (int)L.nc;
  const T* xs = L.x + k * ld;
  const T xc = xs[c];
  T acc = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    const int o = L.nbt[sl * nc + c];
    if (o < 0) continue;
    acc += L.alpha[(sl * S + k) * ld + c] * (xc - xs[o]);
  }
  if (L.tau) {
    const T xm = (k > 0) ? L.x[(k - 1) * ld + c] : (T)0;
    const T xp = (k < S - 1) ? L.x[(k + 1) * ld + c] : (T)0;
    acc += L.tau[k * ld + c] * (2 * xc - xm - xp);
  }
  return acc;
}

// Point update of cell c in slice k of a staged level with tables (point_gs / point_gs_mode).
template <typename T, int MODE>
__device__ __forceinline__ void point_gs_t(int S, const LevelView<T>& L, const LevelView<T>& Lc, int k, int c) {
  const int ld = (int)L.ld, nc = (int)L.nc;
  T num = L.b[k * ld + c], den = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    const T a = L.alpha[(sl * S + k) * ld + c];
    den += a;
    const int o = L.nbt[sl * nc + c];
    if (MODE != kSweepFromZero && o >= 0) num += a * sweep_neighbour_t<T, MODE>(L, Lc, k, o);
  }
  L.x[k * ld + c] = mg_div(num, den);
}

// Line update of cell c (same system as line_gs) by one warp; neighbour
// values as the sweep mode gives them.
template <typename T, int KPL, int MODE>
__device__ __forceinline__ void line_pcr_mode(int S, const LevelView<T>& L, const LevelView<T>& Lc, i64 c, int lane) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  T a[KPL], d[KPL], cc[KPL], r[KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    int k = lane + 32 * q;
    if (k < S) {
      i64 o = (i64)k * L.ld;
      T tau = L.tau[o + c];
      T dg = 2 * tau, rhs = L.b[o + c];
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        T al = L.alpha[((i64)sl * S + k) * L.ld + c];
        dg += al;
        if (MODE != kSweepFromZero && nb[sl] >= 0) rhs += al * sweep_neighbour<T, MODE>(L, Lc, k, (int)nb[sl]);
      }
      d[q] = dg;
      r[q] = rhs;
      a[q] = (k > 0) ? -tau : (T)0;
      cc[q] = (k < S - 1) ? -tau : (T)0;
    } else {
      d[q] = 1; r[q] = 0; a[q] = 0; cc[q] = 0;
    }
  }
  pcr_solve<T, KPL>(a, d, cc, r, lane);
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    int k = lane + 32 * q;
    if (k < S) L.x[(i64)k * L.ld + c] = mg_div(r[q], d[q]);
  }
}

template <typename T, int KPL>
__device__ __forceinline__ void line_pcr(int S, const LevelView<T>& L, i64 c, int lane) {
  line_pcr_mode<T, KPL, kSweepPlain>(S, L, L, c, lane);
}

// Point update of cell c in slice k with the sweep mode's neighbour values.
template <typename T, int MODE>
__device__ __forceinline__ void point_gs_mode(int S, const LevelView<T>& L, const LevelView<T>& Lc, int k, int c) {
  i64 nb[3];
  neighbours(L.m, decode(L.m, c), nb);
  T num = L.b[(i64)k * L.ld + c], den = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    T a = L.alpha[((i64)sl * S + k) * L.ld + c];
    den += a;
    if (MODE != kSweepFromZero && nb[sl] >= 0) num += a * sweep_neighbour<T, MODE>(L, Lc, k, (int)nb[sl]);
  }
  L.x[(i64)k * L.ld + c] = mg_div(num, den);
}

// Point sweep of one colour laid out by rows of squares: warp w of the CTA
// takes row J = blockIdx.x * 8 + w, its lanes the squares I of that row, so
// the cell and its three neighbours follow from (t, I, J) without a division
// and every load of a row is coalesced.  The same operations in the same
// order as point_gs / point_gs_mode.
template <typename T>
__device__ __forceinline__ int parent_cell(int m, int t, int I, int J) {
  const int n = m >> 1, a = I & 1, b = J & 1;
  const int tc = (t == 0) ? ((a == 0 && b == 1) ? 1 : 0) : ((a == 1 && b == 0) ? 0 : 1);
  return tc * n * n + (J >> 1) * n + (I >> 1);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_point_rows_kernel(int S, LevelView<T> L, LevelView<T> Lc, int color) {
  OT_GRID_DEP_WAIT();
  const int m = L.m, mm = m * m, ld = (int)L.ld;
  const int J = blockIdx.x * 8 + threadIdx.y;
  if (J >= m) return;
  const int t = color, to = 1 - color;
  for (int k = blockIdx.y; k < S; k += gridDim.y) {
    const T* xs = L.x + k * ld;
    const T* xcs = (MODE == kSweepAfterProlong) ? Lc.x + k * (int)Lc.ld : nullptr;
    for (int I = threadIdx.x; I < m; I += 32) {
      const int c = t * mm + J * m + I;
      // neighbours (slot 0, 1, 2) as (I, J) of the other triangle type
      int nI[3], nJ[3];
      bool has[3];
      nI[0] = I, nJ[0] = J, has[0] = true;
      if (t == 0) {
        nI[1] = I + 1, nJ[1] = J, has[1] = I + 1 < m;
        nI[2] = I, nJ[2] = J - 1, has[2] = J > 0;
      } else {
        nI[1] = I - 1, nJ[1] = J, has[1] = I > 0;
        nI[2] = I, nJ[2] = J + 1, has[2] = J + 1 < m;
      }
      T num = L.b[k * ld + c], den = 0;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        T a = L.alpha[(sl * S + k) * ld + c];
        den += a;
        if (MODE != kSweepFromZero && has[sl]) {
          T v = xs[to * mm + nJ[sl] * m + nI[sl]];
          if (MODE == kSweepAfterProlong) v += xcs[parent_cell<T>(m, to, nI[sl], nJ[sl])];
          num += a * v;
        }
      }
      L.x[k * ld + c] = mg_div(num, den);
    }
  }
}

// Rows kernel usable: 32-bit indices over the level.
template <typename T>
static bool point_rows_ok(int S, const LevelView<T>& L) {
  return 3 * (i64)S * L.ld < (1ll << 31);
}

template <typename T, int MODE>
static void launch_point_rows(int S, const LevelView<T>& L, const LevelView<T>& Lc, int color, Stream st) {
  const dim3 grid((unsigned)((L.m + 7) / 8), (unsigned)(S < 65535 ? S : 65535));
  launch(k_point_rows_kernel<T, MODE>, grid, dim3(32, 8), 0, cs(st), S, L, Lc, color);
}

template <typename T, int KPL>
__global__ void __launch_bounds__(256) k_line_pcr_kernel(int S, LevelView<T> L, int color) {
  OT_GRID_DEP_WAIT();
  i64 sq = (i64)L.m * L.m;
  int lane = threadIdx.x & 31;
  i64 w0 = (blockIdx.x * (i64)blockDim.x + threadIdx.x) >> 5;
  i64 nw = ((i64)gridDim.x * blockDim.x) >> 5;
  for (i64 w = w0; w < sq; w += nw) line_pcr<T, KPL>(S, L, (i64)color * sq + w, lane);
}

static inline int pcr_kpl(int S) { return S <= 32 ? 1 : (S <= 64 ? 2 : (S <= 128 ? 4 : 0)); }

// Tiled line smoother: a CTA of TC warps owns TC consecutive cells of one
// colour.  Their K-slice systems are gathered with row loads of TC cells into
// a padded [K][TC+1] shared tile (each thread loads its KPL rows before using
// any), warp w solves column w through the line's stored Thomas factors, and
// the solutions leave through the same tile.  TC = 8 keeps many CTAs on small
// levels; TC = 16 gives 64-byte row segments (FP32) on large ones.  The stages
// of one tile are run by the 32 TC threads (tid) of a CTA on their own shared
// tile (3 S (TC+1) values), with a barrier between stages.  tile: index of the
// first cell / TC.
template <typename T, int TC, int KPL>
__device__ __forceinline__ void tile_store(int S, const LevelView<T>& L, int color, int tile, int tid, const T* tsm) {
  constexpr int P = TC + 1;
  const T* sr = tsm + S * P;
  const int sq = L.m * L.m, ld = (int)L.ld;
  const int j = tid % TC, row0 = tid / TC;
  const int cell = tile * TC + j;
  if (cell < sq) {
#pragma unroll
    for (int q = 0; q < KPL; ++q) {
      const int k = row0 + 32 * q;
      if (k < S) L.x[k * ld + color * sq + cell] = sr[k * P + j];
    }
  }
}

// Thomas factors of every line of a level in device memory (once per Newton step).
template <typename T>
__global__ void k_line_factor_kernel(int S, LevelView<T> L) {
  OT_GRID_DEP_WAIT();
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)L.nc; c += gridDim.x * blockDim.x) line_factor(S, L, c);
}

template <typename T>
void k_mg_line_factor(int S, const LevelView<T>& L, Stream st) {
  if (!L.fac || !L.tau) return;
  launch(k_line_factor_kernel<T>, nblk(L.nc), kT, 0, cs(st), S, L);
}

// The tile stages with stored factors: the gather writes the substitution
// coefficients A = tau/den, B = r/den, C = -cp (r: the line's right-hand side
// with the neighbour values of the sweep mode), the solve runs scan_tridiag on
// contiguous rows per lane.
template <typename T, int TC, int KPL, int MODE>
__device__ __forceinline__ void tile_gather_fac(int S, const LevelView<T>& L, const LevelView<T>& Lc, int color,
                                                int tile, int tid, T* tsm) {
  constexpr int P = TC + 1;
  T* sa = tsm;
  T* sb = sa + S * P;
  T* sc = sb + S * P;
  const int sq = L.m * L.m, ld = (int)L.ld;
  const int j = tid % TC, row0 = tid / TC;
  const int cell = tile * TC + j;
  const bool live = cell < sq;
  i64 nb[3] = {-1, -1, -1};
  const int c = color * sq + cell;
  if (live) neighbours(L.m, decode(L.m, c), nb);
  const T* inv = L.fac;
  const T* cpf = L.fac + (i64)S * ld;
  T tau[KPL], bb[KPL], iv[KPL], cp[KPL], al[KPL][3], xn[KPL][3];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = row0 + 32 * q;
    tau[q] = 0, bb[q] = 0, iv[q] = 0, cp[q] = 0;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) al[q][sl] = 0, xn[q][sl] = 0;
    if (live && k < S) {
      const int o = k * ld + c;
      tau[q] = L.tau[o];
      bb[q] = L.b[o];
      iv[q] = inv[o];
      cp[q] = cpf[o];
      if (MODE != kSweepFromZero) {
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
          al[q][sl] = L.alpha[(sl * S + k) * ld + c];
          if (nb[sl] >= 0) xn[q][sl] = sweep_neighbour<T, MODE>(L, Lc, k, (int)nb[sl]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = row0 + 32 * q;
    if (k >= S) continue;
    T rhs = bb[q];
    if (MODE != kSweepFromZero) {
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) rhs += al[q][sl] * xn[q][sl];
    }
    sa[k * P + j] = (k > 0) ? tau[q] * iv[q] : (T)0;
    sb[k * P + j] = rhs * iv[q];
    sc[k * P + j] = -cp[q];
  }
}

template <typename T, int TC, int KPL>
__device__ __forceinline__ void tile_solve_fac(int S, int tid, T* tsm) {
  constexpr int P = TC + 1;
  T* sa = tsm;
  T* sb = sa + S * P;
  T* sc = sb + S * P;
  const int lane = tid & 31, col = tid >> 5;
  T A[KPL], B[KPL], C[KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = lane * KPL + q;
    const bool in = k < S;
    A[q] = in ? sa[k * P + col] : (T)0;
    B[q] = in ? sb[k * P + col] : (T)0;
    C[q] = in ? sc[k * P + col] : (T)0;
  }
  __syncwarp();
  scan_tridiag<T, KPL>(A, B, C, lane);
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = lane * KPL + q;
    if (k < S) sb[k * P + col] = B[q];
  }
}

template <typename T, int TC, int KPL, int MODE>
__global__ void __launch_bounds__(32 * TC) k_line_scan_tile_kernel(int S, LevelView<T> L, LevelView<T> Lc, int color) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tsm = reinterpret_cast<T*>(smem_raw);
  tile_gather_fac<T, TC, KPL, MODE>(S, L, Lc, color, blockIdx.x, threadIdx.x, tsm);
  __syncthreads();
  tile_solve_fac<T, TC, KPL>(S, threadIdx.x, tsm);
  __syncthreads();
  tile_store<T, TC, KPL>(S, L, color, blockIdx.x, threadIdx.x, tsm);
}

// Cells per tile of the line smoother for a level of sq cells per colour.
static inline int tile_cells(i64 sq) { return sq >= 16384 ? 16 : 8; }

template <typename T, int TC, int MODE>
static void launch_tile_tc(int S, const LevelView<T>& L, const LevelView<T>& Lc, int color, int kpl, Stream st) {
  const i64 sq = (i64)L.m * L.m;
  const int blocks = (int)((sq + TC - 1) / TC);
  const size_t tile = 3 * (size_t)S * (TC + 1) * sizeof(T);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(st);
  if (kpl == 1)
    launch(k_line_scan_tile_kernel<T, TC, 1, MODE>, blocks, 32 * TC, tile, s, S, L, Lc, color);
  else if (kpl == 2)
    launch(k_line_scan_tile_kernel<T, TC, 2, MODE>, blocks, 32 * TC, tile, s, S, L, Lc, color);
  else
    launch(k_line_scan_tile_kernel<T, TC, 4, MODE>, blocks, 32 * TC, tile, s, S, L, Lc, color);
}

// The tile width for this shape, or 0 if no tiled sweep applies (no stored line
// factors, K > 128, a tile beyond 48 KB of shared memory, or indices beyond 32 bits).
template <typename T>
static int tile_width(int S, const LevelView<T>& L) {
  if (!L.fac) return 0;
  int tc = tile_cells((i64)L.m * L.m);
  if (3 * (size_t)S * (tc + 1) * sizeof(T) > 48 * 1024) tc = 8;
  if (pcr_kpl(S) == 0 || 3 * (size_t)S * (tc + 1) * sizeof(T) > 48 * 1024 || 3 * (i64)S * L.ld >= (1ll << 31)) return 0;
  return tc;
}

// The tiled line sweep of one colour in a mode, if the shape allows one; false otherwise.
template <typename T, int MODE>
static bool launch_tile(int S, const LevelView<T>& L, const LevelView<T>& Lc, int color, Stream st) {
  const int kpl = pcr_kpl(S);
  const int tc = tile_width(S, L);
  if (tc == 0) return false;
  if (tc == 16)
    launch_tile_tc<T, 16, MODE>(S, L, Lc, color, kpl, st);
  else
    launch_tile_tc<T, 8, MODE>(S, L, Lc, color, kpl, st);
  return true;
}

// Opt a kernel into more than 48 KB of dynamic shared memory (once per size).
template <typename Kern>
static void set_smem(Kern k, size_t bytes) {
  static std::unordered_map<const void*, size_t> granted;
  static std::mutex guard;  // concurrent solves share this table
  if (bytes <= 48 * 1024) return;
  std::lock_guard<std::mutex> lock(guard);
  size_t& g = granted[reinterpret_cast<const void*>(k)];
  if (bytes <= g) return;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) throw Error(7, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  g = bytes;
}

template <typename T>
void k_mg_smooth(int S, const LevelView<T>& L, int color, T* line_c, T* line_r, Stream st) {
  i64 sq = (i64)L.m * L.m;
  int id = L.tau ? prof::SCH_SMOOTH : prof::LAP_SMOOTH;
  prof::begin(id, st);
  if (L.tau) {
    int kpl = pcr_kpl(S);
    if (launch_tile<T, kSweepPlain>(S, L, L, color, st)) {
      prof::end(id, st, (double)sizeof(T) * 7.0 * (double)S * (double)sq);
      return;
    }
    int blocks = (int)std::min<i64>((sq * 32 + kT - 1) / kT, 1 << 20);
    if (kpl == 1)
      launch(k_line_pcr_kernel<T, 1>, blocks, kT, 0, cs(st), S, L, color);
    else if (kpl == 2)
      launch(k_line_pcr_kernel<T, 2>, blocks, kT, 0, cs(st), S, L, color);
    else if (kpl == 4)
      launch(k_line_pcr_kernel<T, 4>, blocks, kT, 0, cs(st), S, L, color);
    else
      launch(k_line_smooth_kernel<T>, nblk(sq), kT, 0, cs(st), S, L, color, line_c, line_r);
  } else {
    if (point_rows_ok(S, L))
      launch_point_rows<T, kSweepPlain>(S, L, L, color, st);
    else
      launch(k_point_smooth_kernel<T>, slice_grid(sq, S), kT, 0, cs(st), S, L, color);
  }
  // per updated cell: b, three coefficients, the neighbours' x, the new x (+ tau for lines)
  prof::end(id, st, (double)sizeof(T) * (L.tau ? 7.0 : 6.0) * (double)S * (double)sq);
}

template <typename T, int MODE>
__global__ void k_point_smooth_mode_kernel(int S, LevelView<T> L, LevelView<T> Lc, int color) {
  OT_GRID_DEP_WAIT();
  const int sq = L.m * L.m;
  SLICE_LOOP(k, S, i, sq) point_gs_mode<T, MODE>(S, L, Lc, k, color * sq + (int)i);
}

template <typename T>
void k_mg_smooth_mode(int S, const LevelView<T>& L, const LevelView<T>* coarse, int color, int mode, T* line_c,
                      T* line_r, Stream st) {
  if (mode == kSweepPlain) {
    k_mg_smooth<T>(S, L, color, line_c, line_r, st);
    return;
  }
  if (mode == kSweepAfterProlong && !coarse) throw Error(1, "sweep after prolongation needs the coarse level");
  const LevelView<T> Lc = coarse ? *coarse : L;
  const i64 sq = (i64)L.m * L.m;
  const int id = L.tau ? prof::SCH_SMOOTH : prof::LAP_SMOOTH;
  if (L.tau && tile_width(S, L) == 0) {
    // no tiled kernel for this shape: make the mode explicit, then a plain sweep
    if (mode == kSweepFromZero)
      dev::zero(L.x, sizeof(T) * (size_t)S * L.ld, st);
    else
      k_mg_prolong<T>(S, Lc, L, st);
    k_mg_smooth<T>(S, L, color, line_c, line_r, st);
    return;
  }
  prof::begin(id, st);
  if (L.tau) {
    if (mode == kSweepFromZero)
      launch_tile<T, kSweepFromZero>(S, L, Lc, color, st);
    else
      launch_tile<T, kSweepAfterProlong>(S, L, Lc, color, st);
  } else if (mode == kSweepFromZero) {
    if (point_rows_ok(S, L))
      launch_point_rows<T, kSweepFromZero>(S, L, Lc, color, st);
    else
      launch(k_point_smooth_mode_kernel<T, kSweepFromZero>, slice_grid(sq, S), kT, 0, cs(st), S, L, Lc, color);
  } else {
    if (point_rows_ok(S, L))
      launch_point_rows<T, kSweepAfterProlong>(S, L, Lc, color, st);
    else
      launch(k_point_smooth_mode_kernel<T, kSweepAfterProlong>, slice_grid(sq, S), kT, 0, cs(st), S, L, Lc, color);
  }
  prof::end(id, st, (double)sizeof(T) * (L.tau ? 7.0 : 6.0) * (double)S * (double)sq);
}

// ------------------------------------------------------------------ residual and transfers
template <typename T>
__global__ void k_residual_kernel(int S, LevelView<T> L) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k, S, c, L.nc) {
    i64 i = (i64)k * L.ld + c;
    L.r[i] = L.b[i] - level_apply(S, L, k, c);
  }
}

template <typename T>
void k_mg_residual(int S, const LevelView<T>& L, Stream st) {
  prof::begin(prof::MG_TRANSFER, st);
  launch(k_residual_kernel<T>, slice_grid(L.nc, S), kT, 0, cs(st), S, L);
  prof::end(prof::MG_TRANSFER, st, (double)sizeof(T) * (L.tau ? 7.0 : 6.0) * (double)S * (double)L.nc);
}

template <typename T>
__global__ void k_restrict_kernel(int S, LevelView<T> f, LevelView<T> c) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k, S, C, c.nc) {
    i64 i = (i64)k * c.ld + C;
    i64 ch[4];
    children(c.m, decode(c.m, C), ch);
    const T* rf = f.r + (i64)k * f.ld;
    c.b[i] = rf[ch[0]] + rf[ch[1]] + rf[ch[2]] + rf[ch[3]];
  }
}

template <typename T>
void k_mg_restrict(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st) {
  launch(k_restrict_kernel<T>, slice_grid(coarse.nc, S), kT, 0, cs(st), S, fine, coarse);
}

// b_coarse = J^T (b - M x) without storing the fine residual: each coarse cell
// sums its four children's residuals (same sums, same order as residual + restrict).
template <typename T>
__global__ void k_restrict_residual_kernel(int S, LevelView<T> f, LevelView<T> c) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k, S, C, c.nc) {
    i64 ch[4];
    children(c.m, decode(c.m, C), ch);
    const T* bf = f.b + (i64)k * f.ld;
    T acc = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) acc += bf[ch[a]] - level_apply(S, f, k, ch[a]);
    c.b[(i64)k * c.ld + C] = acc;
  }
}

// level_apply for fine triangle (t, I, J) in the row layout (32-bit indices).
template <typename T>
__device__ __forceinline__ T level_apply_row(int S, const LevelView<T>& L, int k, int t, int I, int J) {
  const int m = L.m, ld = (int)L.ld;
  const int c = t * m * m + J * m + I;
  const T* xs = L.x + k * ld;
  const T xc = xs[c];
  T acc = 0;
#pragma unroll
  for (int sl = 0; sl < 3; ++sl) {
    int Io, Jo;
    const int o = row_nb(m, t, I, J, sl, &Io, &Jo);
    if (o < 0) continue;
    acc += L.alpha[(sl * S + k) * ld + c] * (xc - xs[o]);
  }
  if (L.tau) {
    const T xm = (k > 0) ? L.x[(k - 1) * ld + c] : (T)0;
    const T xp = (k < S - 1) ? L.x[(k + 1) * ld + c] : (T)0;
    acc += L.tau[k * ld + c] * (2 * xc - xm - xp);
  }
  return acc;
}

// b_coarse = J^T (b - M x) with a warp per row of coarse squares (as k_restrict_residual_kernel).
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_residual_rows(int S, LevelView<T> f, LevelView<T> c) {
  OT_GRID_DEP_WAIT();
  const int n = c.m, nn = n * n, m = f.m, mm = m * m, fld = (int)f.ld, cld = (int)c.ld;
  const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y;
  if (i >= n || j >= n) return;
  for (int k = blockIdx.z; k < S; k += gridDim.z) {
    const T* bf = f.b + k * fld;
    for (int t = 0; t < 2; ++t) {
      int ct[4], cI[4], cJ[4];
      row_children(t, i, j, ct, cI, cJ);
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) acc += bf[ct[a] * mm + cJ[a] * m + cI[a]] - level_apply_row(S, f, k, ct[a], cI[a], cJ[a]);
      c.b[k * cld + t * nn + j * n + i] = acc;
    }
  }
}

template <typename T>
void k_mg_restrict_residual(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st) {
  prof::begin(prof::MG_TRANSFER, st);
  if (point_rows_ok(S, fine) && point_rows_ok(S, coarse)) {
    const dim3 grid((unsigned)((coarse.m + 31) / 32), (unsigned)((coarse.m + 7) / 8), (unsigned)(S < 65535 ? S : 65535));
    launch(k_restrict_residual_rows<T>, grid, dim3(32, 8), 0, cs(st), S, fine, coarse);
  } else {
    launch(k_restrict_residual_kernel<T>, slice_grid(coarse.nc, S), kT, 0, cs(st), S, fine, coarse);
  }
  prof::end(prof::MG_TRANSFER, st, (double)sizeof(T) * (fine.tau ? 6.0 : 5.0) * (double)S * (double)fine.nc);
}

template <typename T>
__global__ void k_prolong_kernel(int S, LevelView<T> c, LevelView<T> f) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k, S, cf, f.nc) f.x[(i64)k * f.ld + cf] += c.x[(i64)k * c.ld + parent_of(f.m, cf)];
}

template <typename T>
void k_mg_prolong(int S, const LevelView<T>& coarse, const LevelView<T>& fine, Stream st) {
  launch(k_prolong_kernel<T>, slice_grid(fine.nc, S), kT, 0, cs(st), S, coarse, fine);
}

// ------------------------------------------------------------------ coarsest grid
// Walks the (slice, cell) pairs k nc + c of S nc cells in steps of blockDim.x
// with one division per thread and level: (k, c) advance by (dk, dc).
struct SliceWalk {
  int k, c, dk, dc, nc;
  __device__ SliceWalk(int nc_) : nc(nc_) {
    k = threadIdx.x / nc;
    c = threadIdx.x - k * nc;
    dk = blockDim.x / nc;
    dc = blockDim.x - dk * nc;
  }
  __device__ void next() {
    k += dk;
    c += dc;
    if (c >= nc) {
      c -= nc;
      ++k;
    }
  }
};

// ---- time lines with stored Thomas factors (fused shared-memory levels).
// Row k of the line of cell c: d_k x_k - tau_k (x_{k-1} + x_{k+1}) = r_k with
// d_k = 2 tau_k + sum_slot alpha, x_{-1} = x_S = 0 (the system line_gs solves).
// line_factor stores 1/den_k and cp_k = -tau_k/den_k of the forward
// elimination, den_0 = d_0, den_k = d_k + tau_k cp_{k-1}; a sweep then needs
// one multiply-add per row forward and one back.
template <typename T>
__device__ __forceinline__ void line_factor(int S, const LevelView<T>& L, int c) {
  const i64 ld = L.ld;
  T* inv = L.fac;
  T* cp = L.fac + (i64)S * ld;
  T cprev = 0;
  for (int k = 0; k < S; ++k) {
    const i64 o = (i64)k * ld + c;
    const T tau = L.tau[o];
    T dg = 2 * tau;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) dg += L.alpha[((i64)sl * S + k) * ld + c];
    const T den = dg + (k > 0 ? tau * cprev : (T)0);
    const T iv = mg_div((T)1, den);
    inv[o] = iv;
    cprev = (k < S - 1) ? -tau * iv : (T)0;
    cp[o] = cprev;
  }
}

// One line of a staged level by one warp with the stored factors: the lanes
// form their rows' right-hand sides b + sum_slot alpha x_neighbour (neighbour
// values as the sweep mode gives them) in parallel, then scan_tridiag.
template <typename T, int KPL, int MODE>
__device__ __forceinline__ void line_scan_solve(int S, const LevelView<T>& L, const LevelView<T>& Lc, int c,
                                                int lane) {
  int nb[3];
  if (L.nbt) {
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) nb[sl] = L.nbt[sl * (int)L.nc + c];
  } else {
    i64 nl[3];
    neighbours(L.m, decode(L.m, c), nl);
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) nb[sl] = (int)nl[sl];
  }
  const int ld = (int)L.ld;
  const T* inv = L.fac;
  const T* cp = L.fac + S * ld;
  T A[KPL], B[KPL], C[KPL];
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = lane * KPL + q;
    A[q] = 0;
    B[q] = 0;
    C[q] = 0;
    if (k < S) {
      const int o = k * ld + c;
      T rhs = L.b[o];
      if (MODE != kSweepFromZero) {
#pragma unroll
        for (int sl = 0; sl < 3; ++sl)
          if (nb[sl] >= 0)
            rhs += L.alpha[(sl * S + k) * ld + c] *
                   (L.par ? sweep_neighbour_t<T, MODE>(L, Lc, k, nb[sl]) : sweep_neighbour<T, MODE>(L, Lc, k, nb[sl]));
      }
      const T iv = inv[o];
      A[q] = (k > 0) ? L.tau[o] * iv : (T)0;
      B[q] = rhs * iv;
      C[q] = -cp[o];
    }
  }
  scan_tridiag<T, KPL>(A, B, C, lane);
#pragma unroll
  for (int q = 0; q < KPL; ++q) {
    const int k = lane * KPL + q;
    if (k < S) L.x[k * ld + c] = B[q];
  }
}

// One colour sweep of a staged level: warp w of the CTA takes lines w, w + nwarp, ...
template <typename T, int KPL, int MODE>
__device__ void line_scan_sweep(int S, const LevelView<T>& L, const LevelView<T>& Lc, int color) {
  const int sq = L.m * L.m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int w = warp; w < sq; w += nwarp) line_scan_solve<T, KPL, MODE>(S, L, Lc, color * sq + w, lane);
}

// Threads of the one-CTA Schur kernels: 512 where a PCR lane's KPL systems in T
// would not fit the 64 registers a 1024-thread CTA leaves each thread.
template <typename T, int KPL>
constexpr int sch_lower_threads() {
  return sizeof(T) * KPL >= 16 ? 512 : 1024;
}

// One CTA: x = 0, `sweeps` red-black sweeps; for the space-time operator also
// the correction on the single aggregate of all cells (the Galerkin operator
// on the constant-per-slice space is the time-tridiagonal tau_G (2 d^k - d^{k-1} - d^{k+1}),
// tau_G = sum of tau over the cells), followed by `sweeps` more sweeps.  A
// space-time level of side 1 is solved exactly instead.
// KPL > 0: time lines and the aggregate system by warp PCR; KPL = 0: Thomas per thread.
template <typename T, int KPL>
__device__ void coarse_body(int S, const LevelView<T>& L, int sweeps, T* lc, T* lr, T* agg) {
  if (L.tau && L.m == 1) {
    if (threadIdx.x == 0) coarse_exact_side1(S, L, agg);
    __syncthreads();
    return;
  }
  const int sq = L.m * L.m, nc = (int)L.nc;
  const i64 ld = L.ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (SliceWalk w(nc); w.k < S; w.next()) L.x[w.k * ld + w.c] = 0;
  __syncthreads();
  int passes = L.tau ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    for (int it = 0; it < sweeps; ++it) {
      for (int color = 0; color < 2; ++color) {
        if (L.tau && L.fac && KPL > 0) {
          line_scan_sweep<T, (KPL > 0 ? KPL : 1), kSweepPlain>(S, L, L, color);
        } else if (L.tau && KPL > 0) {
          for (int w = warp; w < sq; w += nwarp) line_pcr<T, (KPL > 0 ? KPL : 1)>(S, L, (i64)color * sq + w, lane);
        } else if (L.tau) {
          for (int i = threadIdx.x; i < sq; i += blockDim.x) line_gs(S, L, (i64)color * sq + i, lc, lr);
        } else {
          for (SliceWalk w(sq); w.k < S; w.next()) point_gs(S, L, w.k, (i64)color * sq + w.c);
        }
        __syncthreads();
      }
    }
    if (!L.tau || pass == passes - 1) break;
    // aggregate correction
    for (SliceWalk w(nc); w.k < S; w.next()) L.r[w.k * ld + w.c] = L.b[w.k * ld + w.c] - level_apply(S, L, w.k, w.c);
    __syncthreads();
    // agg[0..S): rhs, agg[S..2S): tau_G, agg[2S..3S): cp, agg[3S..4S): solution
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
      T rsum = 0, tsum = 0;
      for (int c = 0; c < nc; ++c) {
        rsum += L.r[k * ld + c];
        tsum += L.tau[k * ld + c];
      }
      agg[k] = rsum;
      agg[S + k] = tsum;
    }
    __syncthreads();
    if (KPL > 0) {
      constexpr int Q = KPL > 0 ? KPL : 1;
      if (warp == 0) {
        T a[Q], d[Q], c[Q], r[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          int k = lane + 32 * q;
          if (k < S) {
            T tg = agg[S + k];
            d[q] = 2 * tg;
            r[q] = agg[k];
            a[q] = (k > 0) ? -tg : (T)0;
            c[q] = (k < S - 1) ? -tg : (T)0;
          } else {
            d[q] = 1; r[q] = 0; a[q] = 0; c[q] = 0;
          }
        }
        pcr_solve<T, Q>(a, d, c, r, lane);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          int k = lane + 32 * q;
          if (k < S) agg[3 * S + k] = mg_div(r[q], d[q]);
        }
      }
    } else if (threadIdx.x == 0) {
      T cp = 0, rp = 0;
      for (int k = 0; k < S; ++k) {
        T off = -agg[S + k], dg = 2 * agg[S + k];
        T sub = (k > 0) ? off : (T)0;
        T den = dg - sub * cp;
        cp = (k < S - 1) ? off / den : (T)0;
        rp = (agg[k] - sub * rp) / den;
        agg[2 * S + k] = cp;
        agg[3 * S + k] = rp;
      }
      T xn = 0;
      for (int k = S - 1; k >= 0; --k) {
        T v = agg[3 * S + k] - agg[2 * S + k] * xn;
        agg[3 * S + k] = v;
        xn = v;
      }
    }
    __syncthreads();
    for (SliceWalk w(nc); w.k < S; w.next()) L.x[w.k * ld + w.c] += agg[3 * S + w.k];
    __syncthreads();
  }
}

template <typename T, int KPL>
__global__ void __launch_bounds__(sch_lower_threads<T, KPL>()) k_coarse_kernel(int S, LevelView<T> L, int sweeps,
                                                                                T* lc, T* lr, T* agg) {
  OT_GRID_DEP_WAIT();
  coarse_body<T, KPL>(S, L, sweeps, lc, lr, agg);
}

template <typename T>
void k_mg_coarse_solve(int S, const LevelView<T>& L, int sweeps, T* line_c, T* line_r, T* agg, Stream st) {
  int kpl = L.tau ? pcr_kpl(S) : 0;
  if (kpl == 1)
    launch(k_coarse_kernel<T, 1>, 1, sch_lower_threads<T, 1>(), 0, cs(st), S, L, sweeps, line_c, line_r, agg);
  else if (kpl == 2)
    launch(k_coarse_kernel<T, 2>, 1, sch_lower_threads<T, 2>(), 0, cs(st), S, L, sweeps, line_c, line_r, agg);
  else if (kpl == 4)
    launch(k_coarse_kernel<T, 4>, 1, sch_lower_threads<T, 4>(), 0, cs(st), S, L, sweeps, line_c, line_r, agg);
  else
    launch(k_coarse_kernel<T, 0>, 1, sch_lower_threads<T, 0>(), 0, cs(st), S, L, sweeps, line_c, line_r, agg);
}

// ------------------------------------------------------------------ fused lower levels
// The small levels of a V-cycle (from levels[0] down to the coarsest) in one
// launch, staged in shared memory: the CTA copies every fused level's
// coefficients and the first level's right-hand side in, runs the same
// operations in the same order as the per-level kernels with block barriers
// between phases, and writes the first level's x back.
template <typename T>
struct LevelSet {
  int n;
  LevelView<T> L[16];
};

// Slice stride of a staged level: odd when S_view > 1, so that a warp reading
// one cell's time line (lane = slice) touches 32 different banks.
__host__ __device__ inline i64 staged_ld(i64 nc, int S_view) { return (S_view > 1 && (nc & 1) == 0) ? nc + 1 : nc; }

// One element global -> shared without a register round trip (cp.async): a
// thread issues all its copies back to back and waits once (async_copy_wait),
// instead of one L2 round trip per element.
template <typename T>
__device__ __forceinline__ void async_copy_elem(T* sdst, const T* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void async_copy_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Carve shared-memory views of the fused levels (S_view slices each) and copy
// coefficients (slice `slice0` onwards) and the first level's b into them.
template <typename T>
__device__ void stage_levels(const LevelSet<T>& g, LevelSet<T>& s, T* smem, int S, int S_view, int slice0) {
  if (threadIdx.x == 0) {
    T* p = smem;
    s.n = g.n;
    for (int l = 0; l < g.n; ++l) {
      const LevelView<T>& G = g.L[l];
      LevelView<T>& V = s.L[l];
      V.m = G.m;
      V.nc = G.nc;
      V.ld = staged_ld(G.nc, S_view);
      const i64 n1 = (i64)S_view * V.ld;
      V.alpha = p;
      p += 3 * n1;
      V.tau = G.tau ? p : nullptr;
      if (G.tau) p += n1;
      V.x = p;
      p += n1;
      V.b = p;
      p += n1;
      V.r = p;
      p += n1;
      V.fac = nullptr;
      if (G.tau) {
        V.fac = p;
        p += 2 * n1;
      }
    }
    if (g.L[g.n - 1].tau) p += 4 * S_view;  // the aggregate scratch after the last level (sch_lower_body)
    int* q = reinterpret_cast<int*>(p);
    for (int l = 0; l < g.n; ++l) {
      LevelView<T>& V = s.L[l];
      const int nc = (int)V.nc;
      V.nbt = q;
      V.par = q + 3 * nc;
      V.chd = q + 4 * nc;
      q += 8 * nc;
    }
  }
  __syncthreads();
  // neighbour, parent and child tables of every staged level (one pass over all cells)
  {
    int total = 0;
    for (int l = 0; l < g.n; ++l) total += (int)s.L[l].nc;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      int l = 0, c = i;
      while (c >= (int)s.L[l].nc) c -= (int)s.L[l++].nc;
      const LevelView<T>& V = s.L[l];
      const int nc = (int)V.nc;
      const Cell q = decode(V.m, c);
      i64 nb[3];
      neighbours(V.m, q, nb);
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) V.nbt[sl * nc + c] = (int)nb[sl];
      V.par[c] = (l + 1 < g.n) ? (int)parent(V.m, q) : -1;
      if (l > 0) {
        i64 ch[4];
        children(V.m, q, ch);
#pragma unroll
        for (int a = 0; a < 4; ++a) V.chd[a * nc + c] = (int)ch[a];
      }
    }
  }
  for (int l = 0; l < g.n; ++l) {
    const LevelView<T>& G = g.L[l];
    const LevelView<T>& V = s.L[l];
    const int nc = (int)G.nc, gld = (int)G.ld, vld = (int)V.ld;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      const T* src = G.alpha + ((i64)sl * S + slice0) * gld;
      T* dst = V.alpha + sl * S_view * vld;
      for (SliceWalk w(nc); w.k < S_view; w.next()) async_copy_elem(dst + w.k * vld + w.c, src + w.k * gld + w.c);
    }
    if (G.tau) {
      const T* src = G.tau + (i64)slice0 * gld;
      for (SliceWalk w(nc); w.k < S_view; w.next()) async_copy_elem(V.tau + w.k * vld + w.c, src + w.k * gld + w.c);
    }
    if (l == 0) {
      const T* src = G.b + (i64)slice0 * gld;
      for (SliceWalk w(nc); w.k < S_view; w.next()) async_copy_elem(V.b + w.k * vld + w.c, src + w.k * gld + w.c);
    }
  }
  async_copy_wait();
  __syncthreads();
}

template <typename T>
size_t fused_smem_bytes(const LevelView<T>* lv, int nlev, int S_view, bool tc) {
  size_t cells = 0;
  for (int l = 0; l < nlev; ++l) cells += (size_t)S_view * (size_t)staged_ld(lv[l].nc, S_view);
  size_t tables = 0;  // neighbour, parent and child tables: 8 ints per cell of every level
  for (int l = 0; l < nlev; ++l) tables += 8 * sizeof(int) * (size_t)lv[l].nc;
  return sizeof(T) * cells * (tc ? 9 : 6) + (tc ? sizeof(T) * 4 * (size_t)S_view : 0) + tables;
}

// Slice Laplacians: one CTA per slice (blockIdx.x), point red-black GS, the
// slice's levels in shared memory (S_view = 1: stride = cells).
constexpr int kLapLowerThreads = 1024;  // one cell per thread and colour phase on a side-32 level
template <typename T>
__global__ void __launch_bounds__(kLapLowerThreads) k_lap_lower_kernel(int S, LevelSet<T> gls, int nu, int nuc) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x;
  __shared__ LevelSet<T> ls;
  stage_levels(gls, ls, reinterpret_cast<T*>(smem_raw), S, 1, k);
  const int last = ls.n - 1;
  // (the first sweep of a level reads zero neighbours, so x needs no reset,
  // except on the coarsest level and when there are no sweeps)
  for (int l = 0; l <= last; ++l) {
    const LevelView<T>& L = ls.L[l];
    const int sq = L.m * L.m, nc = (int)L.nc;
    const int sweeps = (l == last) ? nuc : nu;
    if (sweeps == 0) {
      for (int i = threadIdx.x; i < nc; i += blockDim.x) L.x[i] = 0;
      __syncthreads();
    }
    for (int it = 0; it < sweeps; ++it)
      for (int col = 0; col < 2; ++col) {
        if (it == 0 && col == 0)
          for (int i = threadIdx.x; i < sq; i += blockDim.x) point_gs_t<T, kSweepFromZero>(1, L, L, 0, i);
        else
          for (int i = threadIdx.x; i < sq; i += blockDim.x) point_gs_t<T, kSweepPlain>(1, L, L, 0, col * sq + i);
        __syncthreads();
      }
    if (l == last) break;
    // b_coarse = J^T (b - M x) in one phase
    const LevelView<T>& Lc = ls.L[l + 1];
    const int ncc = (int)Lc.nc;
    for (int C = threadIdx.x; C < ncc; C += blockDim.x) {
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int ch = Lc.chd[a * ncc + C];
        acc += L.b[ch] - level_apply_t(1, L, 0, ch);
      }
      Lc.b[C] = acc;
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= 0; --l) {
    const LevelView<T>& L = ls.L[l];
    const LevelView<T>& Lc = ls.L[l + 1];
    const int sq = L.m * L.m, nc = (int)L.nc;
    if (nu == 0) {
      for (int c = threadIdx.x; c < nc; c += blockDim.x) L.x[c] += Lc.x[L.par[c]];
      __syncthreads();
    }
    for (int it = 0; it < nu; ++it)
      for (int col = 1; col >= 0; --col) {
        if (it == 0 && col == 1)
          for (int i = threadIdx.x; i < sq; i += blockDim.x) point_gs_t<T, kSweepAfterProlong>(1, L, Lc, 0, sq + i);
        else
          for (int i = threadIdx.x; i < sq; i += blockDim.x) point_gs_t<T, kSweepPlain>(1, L, L, 0, col * sq + i);
        __syncthreads();
      }
  }
  const LevelView<T>& G0 = gls.L[0];
  for (int i = threadIdx.x; i < (int)G0.nc; i += blockDim.x) G0.x[(i64)k * G0.ld + i] = ls.L[0].x[i];
}

// Space-time Schur operator: one CTA for all slices, time lines by warp PCR,
// all fused levels in shared memory with odd slice strides; the coarsest level
// as in k_coarse_kernel.
template <typename T, int KPL>
__device__ void sch_lower_body(int S, const LevelSet<T>& gls, int nu, int nuc, unsigned char* smem_raw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  __shared__ LevelSet<T> ls;
  stage_levels(gls, ls, reinterpret_cast<T*>(smem_raw), S, S, 0);
  T* agg = ls.L[ls.n - 1].fac + 2 * (i64)S * ls.L[ls.n - 1].ld;
  const int last = ls.n - 1;
  // the line systems of every staged level, factored once for the whole cycle (one pass over
  // the lines of all levels)
  {
    int total = 0;
    for (int l = 0; l <= last; ++l) total += (int)ls.L[l].nc;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      int l = 0, c = i;
      while (c >= (int)ls.L[l].nc) c -= (int)ls.L[l++].nc;
      line_factor(S, ls.L[l], c);
    }
  }
  __syncthreads();
  for (int l = 0; l < last; ++l) {
    const LevelView<T>& L = ls.L[l];
    const int sq = L.m * L.m, ld = (int)L.ld;
    if (nu == 0) {
      for (int i = threadIdx.x; i < S * ld; i += blockDim.x) L.x[i] = 0;
      __syncthreads();
    }
    for (int it = 0; it < nu; ++it)
      for (int col = 0; col < 2; ++col) {
        if (it == 0 && col == 0)
          line_scan_sweep<T, KPL, kSweepFromZero>(S, L, L, 0);
        else
          line_scan_sweep<T, KPL, kSweepPlain>(S, L, L, col);
        __syncthreads();
      }
    // b_coarse = J^T (b - M x) in one phase
    const LevelView<T>& Lc = ls.L[l + 1];
    const int ldc = (int)Lc.ld;
    const int ncc = (int)Lc.nc;
    for (SliceWalk w(ncc); w.k < S; w.next()) {
      const T* bf = L.b + w.k * ld;
      T acc = 0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int ch = Lc.chd[a * ncc + w.c];
        acc += bf[ch] - level_apply_t(S, L, w.k, ch);
      }
      Lc.b[w.k * ldc + w.c] = acc;
    }
    __syncthreads();
  }
  coarse_body<T, KPL>(S, ls.L[last], nuc, (T*)nullptr, (T*)nullptr, agg);
  __syncthreads();
  for (int l = last - 1; l >= 0; --l) {
    const LevelView<T>& L = ls.L[l];
    const LevelView<T>& Lc = ls.L[l + 1];
    const int sq = L.m * L.m, nc = (int)L.nc, ld = (int)L.ld, ldc = (int)Lc.ld;
    if (nu == 0) {
      for (SliceWalk w(nc); w.k < S; w.next()) L.x[w.k * ld + w.c] += Lc.x[w.k * ldc + L.par[w.c]];
      __syncthreads();
    }
    for (int it = 0; it < nu; ++it)
      for (int col = 1; col >= 0; --col) {
        if (it == 0 && col == 1)
          line_scan_sweep<T, KPL, kSweepAfterProlong>(S, L, Lc, 1);
        else
          line_scan_sweep<T, KPL, kSweepPlain>(S, L, L, col);
        __syncthreads();
      }
  }
  const LevelView<T>& G0 = gls.L[0];
  const LevelView<T>& V0 = ls.L[0];
  for (SliceWalk w((int)G0.nc); w.k < S; w.next()) G0.x[(i64)w.k * G0.ld + w.c] = V0.x[w.k * (int)V0.ld + w.c];
}

template <typename T, int KPL>
__global__ void __launch_bounds__(sch_lower_threads<T, KPL>()) k_sch_lower_kernel(int S, LevelSet<T> gls, int nu,
                                                                                   int nuc) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  sch_lower_body<T, KPL>(S, gls, nu, nuc, smem_raw);
}

template <typename T>
size_t k_mg_fused_smem(int S, const LevelView<T>* levels, int nlev) {
  bool tc = levels[0].tau != nullptr;
  return fused_smem_bytes(levels, nlev, tc ? S : 1, tc);
}

template <typename T>
void k_mg_prepare_lower_cycle(int S, const LevelView<T>* levels, int nlev) {
  const size_t bytes = k_mg_fused_smem(S, levels, nlev);
  if (bytes > kFusedSmemLimit) throw Error(1, "fused multigrid levels exceed shared memory");
  if (!levels[0].tau) {
    set_smem(k_lap_lower_kernel<T>, bytes);
    return;
  }
  const int kpl = pcr_kpl(S);
  if (kpl == 1)
    set_smem(k_sch_lower_kernel<T, 1>, bytes);
  else if (kpl == 2)
    set_smem(k_sch_lower_kernel<T, 2>, bytes);
  else if (kpl == 4)
    set_smem(k_sch_lower_kernel<T, 4>, bytes);
}

template <typename T>
void k_mg_lower_cycle(int S, const LevelView<T>* levels, int nlev, int nu, int nuc, T* line_c, T* line_r, T* agg,
                      Stream st) {
  (void)line_c, (void)line_r, (void)agg;
  if (nlev < 1 || nlev > 16) throw Error(1, "fused multigrid levels out of range");
  LevelSet<T> ls;
  ls.n = nlev;
  for (int i = 0; i < nlev; ++i) ls.L[i] = levels[i];
  const size_t bytes = k_mg_fused_smem(S, levels, nlev);
  if (bytes > kFusedSmemLimit) throw Error(1, "fused multigrid levels exceed shared memory");
  // algorithmic bytes: every fused level's coefficients, the first level's b in and x out
  double moved = 0.0;
  for (int i = 0; i < nlev; ++i) moved += (levels[i].tau ? 4.0 : 3.0) * (double)S * (double)levels[i].nc;
  moved = (double)sizeof(T) * (moved + 2.0 * (double)S * (double)levels[0].nc);
  if (!levels[0].tau) {
    prof::begin(prof::LAP_LOWER, st);
    set_smem(k_lap_lower_kernel<T>, bytes);
    launch(k_lap_lower_kernel<T>, S, kLapLowerThreads, bytes, cs(st), S, ls, nu, nuc);
    prof::end(prof::LAP_LOWER, st, moved);
    return;
  }
  prof::begin(prof::SCH_LOWER, st);
  int kpl = pcr_kpl(S);
  if (kpl == 1) {
    set_smem(k_sch_lower_kernel<T, 1>, bytes);
    launch(k_sch_lower_kernel<T, 1>, 1, sch_lower_threads<T, 1>(), bytes, cs(st), S, ls, nu, nuc);
  } else if (kpl == 2) {
    set_smem(k_sch_lower_kernel<T, 2>, bytes);
    launch(k_sch_lower_kernel<T, 2>, 1, sch_lower_threads<T, 2>(), bytes, cs(st), S, ls, nu, nuc);
  } else if (kpl == 4) {
    set_smem(k_sch_lower_kernel<T, 4>, bytes);
    launch(k_sch_lower_kernel<T, 4>, 1, sch_lower_threads<T, 4>(), bytes, cs(st), S, ls, nu, nuc);
  } else {
    throw Error(1, "fused Schur levels need K <= 128");
  }
  prof::end(prof::SCH_LOWER, st, moved);
}

// ------------------------------------------------------------------ conversions
template <typename T>
__global__ void k_load_kernel(const double* src, double scale, T* b, T* x, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) {
    b[i] = (T)(scale * src[i]);
    if (x) x[i] = 0;
  }
}
template <typename T>
void k_mg_load(const double* src, double scale, T* b, T* x, i64 n, Stream st) {
  launch(k_load_kernel<T>, nblk(n), kT, 0, cs(st), src, scale, b, x, n);
}

template <typename T>
__global__ void k_store_kernel(const T* x, double* dst, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) dst[i] = (double)x[i];
}
template <typename T>
void k_mg_store(const T* x, double* dst, i64 n, Stream st) {
  launch(k_store_kernel<T>, nblk(n), kT, 0, cs(st), x, dst, n);
}

#define OT_INST(T)                                                                                              \
  template void k_mg_lap_coef0<T>(const Dims&, const double*, const double*, const double*, T*, Stream);       \
  template void k_mg_schur_coef0<T>(const Dims&, const double*, const double*, const double*, T*, T*, Stream); \
  template void k_mg_restrict_coef<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                  \
  template void k_mg_smooth<T>(int, const LevelView<T>&, int, T*, T*, Stream);                                 \
  template void k_mg_residual<T>(int, const LevelView<T>&, Stream);                                            \
  template void k_mg_restrict<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                       \
  template void k_mg_restrict_residual<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);              \
  template void k_mg_smooth_mode<T>(int, const LevelView<T>&, const LevelView<T>*, int, int, T*, T*, Stream);  \
  template void k_mg_prolong<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                        \
  template void k_mg_coarse_solve<T>(int, const LevelView<T>&, int, T*, T*, T*, Stream);                       \
  template void k_mg_lower_cycle<T>(int, const LevelView<T>*, int, int, int, T*, T*, T*, Stream);              \
  template void k_mg_prepare_lower_cycle<T>(int, const LevelView<T>*, int);                                    \
  template void k_mg_line_factor<T>(int, const LevelView<T>&, Stream);                                         \
  template size_t k_mg_fused_smem<T>(int, const LevelView<T>*, int);                                           \
  template void k_mg_load<T>(const double*, double, T*, T*, i64, Stream);                                      \
  template void k_mg_store<T>(const T*, double*, i64, Stream);
OT_INST(float)
OT_INST(double)

}  // namespace ot

namespace ot {
template <typename T>
__global__ void k_axpy_t_kernel(const T* x, T a, T* y, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) y[i] += a * x[i];
}
template <typename T>
void k_mg_axpy(const T* x, T a, T* y, i64 n, Stream st) {
  launch(k_axpy_t_kernel<T>, nblk(n), kT, 0, cs(st), x, a, y, n);
}
template void k_mg_axpy<float>(const float*, float, float*, i64, Stream);
template void k_mg_axpy<double>(const double*, double, double*, i64, Stream);
}  // namespace ot
