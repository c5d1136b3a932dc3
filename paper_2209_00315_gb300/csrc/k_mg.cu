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
  int S = d.K + 1;
  i64 tot = (i64)S * d.N;
  GRID_LOOP(i, tot) {
    int jj = (int)(i / d.N);
    i64 c = i - (i64)jj * d.N;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) alpha[((i64)sl * S + jj) * d.N + c] = (T)lap_coef(d, rho, r0, r1, jj, c, sl);
  }
}

template <typename T>
void k_mg_lap_coef0(const Dims& d, const double* rho, const double* r0, const double* r1, T* alpha, Stream st) {
  launch(k_lap_coef0_kernel<T>, nblk((i64)(d.K + 1) * d.N), kT, 0, cs(st), d, rho, r0, r1, alpha);
}

template <typename T>
__global__ void k_schur_coef0_kernel(Dims d, const double* rho, const double* s, T* alpha, T* tau) {
  int S = d.K;
  i64 tot = (i64)S * d.Nc;
  GRID_LOOP(i, tot) {
    int k0 = (int)(i / d.Nc);
    i64 C = i - (i64)k0 * d.Nc;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) alpha[((i64)sl * S + k0) * d.Nc + C] = (T)schur_coef(d, rho, s, k0, C, sl);
    tau[i] = (T)schur_tau(d, rho, k0, C);
  }
}

template <typename T>
void k_mg_schur_coef0(const Dims& d, const double* rho, const double* s, T* alpha, T* tau, Stream st) {
  launch(k_schur_coef0_kernel<T>, nblk((i64)d.K * d.Nc), kT, 0, cs(st), d, rho, s, alpha, tau);
}

// ------------------------------------------------------------------ coarse coefficients
template <typename T>
__global__ void k_restrict_coef_kernel(int S, LevelView<T> f, LevelView<T> c) {
  i64 tot = (i64)S * c.nc;
  GRID_LOOP(i, tot) {
    int k = (int)(i / c.nc);
    i64 C = i - (i64)k * c.nc;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      i64 src[2];
      coarse_coef_sources(c.m, C, sl, src);
      const T* af = f.alpha + ((i64)sl * S + k) * f.nc;
      c.alpha[((i64)sl * S + k) * c.nc + C] = (T)0.5 * (af[src[0]] + af[src[1]]);
    }
    if (c.tau) {
      i64 ch[4];
      children(c.m, decode(c.m, C), ch);
      const T* tf = f.tau + (i64)k * f.nc;
      c.tau[i] = tf[ch[0]] + tf[ch[1]] + tf[ch[2]] + tf[ch[3]];
    }
  }
}

template <typename T>
void k_mg_restrict_coef(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st) {
  launch(k_restrict_coef_kernel<T>, nblk((i64)S * coarse.nc), kT, 0, cs(st), S, fine, coarse);
}

// ------------------------------------------------------------------ smoothers
template <typename T>
__global__ void k_point_smooth_kernel(int S, LevelView<T> L, int color) {
  i64 sq = (i64)L.m * L.m;
  i64 tot = (i64)S * sq;
  GRID_LOOP(i, tot) {
    int k = (int)(i / sq);
    i64 c = (i64)color * sq + (i - (i64)k * sq);
    point_gs(S, L, k, c);
  }
}

template <typename T>
__global__ void k_line_smooth_kernel(int S, LevelView<T> L, int color, T* lc, T* lr) {
  i64 sq = (i64)L.m * L.m;
  GRID_LOOP(i, sq) line_gs(S, L, (i64)color * sq + i, lc, lr);
}

template <typename T>
void k_mg_smooth(int S, const LevelView<T>& L, int color, T* line_c, T* line_r, Stream st) {
  i64 sq = (i64)L.m * L.m;
  int id = L.tau ? prof::SCH_SMOOTH : prof::LAP_SMOOTH;
  prof::begin(id, st);
  if (L.tau)
    launch(k_line_smooth_kernel<T>, nblk(sq), kT, 0, cs(st), S, L, color, line_c, line_r);
  else
    launch(k_point_smooth_kernel<T>, nblk((i64)S * sq), kT, 0, cs(st), S, L, color);
  // per updated cell: b, three coefficients, the neighbours' x, the new x (+ tau for lines)
  prof::end(id, st, (double)sizeof(T) * (L.tau ? 7.0 : 6.0) * (double)S * (double)sq);
}

// ------------------------------------------------------------------ residual and transfers
template <typename T>
__global__ void k_residual_kernel(int S, LevelView<T> L) {
  i64 tot = (i64)S * L.nc;
  GRID_LOOP(i, tot) {
    int k = (int)(i / L.nc);
    L.r[i] = L.b[i] - level_apply(S, L, k, i - (i64)k * L.nc);
  }
}

template <typename T>
void k_mg_residual(int S, const LevelView<T>& L, Stream st) {
  prof::begin(prof::MG_TRANSFER, st);
  launch(k_residual_kernel<T>, nblk((i64)S * L.nc), kT, 0, cs(st), S, L);
  prof::end(prof::MG_TRANSFER, st, (double)sizeof(T) * (L.tau ? 7.0 : 6.0) * (double)S * (double)L.nc);
}

template <typename T>
__global__ void k_restrict_kernel(int S, LevelView<T> f, LevelView<T> c) {
  i64 tot = (i64)S * c.nc;
  GRID_LOOP(i, tot) {
    int k = (int)(i / c.nc);
    i64 C = i - (i64)k * c.nc;
    i64 ch[4];
    children(c.m, decode(c.m, C), ch);
    const T* rf = f.r + (i64)k * f.nc;
    c.b[i] = rf[ch[0]] + rf[ch[1]] + rf[ch[2]] + rf[ch[3]];
  }
}

template <typename T>
void k_mg_restrict(int S, const LevelView<T>& fine, const LevelView<T>& coarse, Stream st) {
  launch(k_restrict_kernel<T>, nblk((i64)S * coarse.nc), kT, 0, cs(st), S, fine, coarse);
}

template <typename T>
__global__ void k_prolong_kernel(int S, LevelView<T> c, LevelView<T> f) {
  i64 tot = (i64)S * f.nc;
  GRID_LOOP(i, tot) {
    int k = (int)(i / f.nc);
    i64 cf = i - (i64)k * f.nc;
    f.x[i] += c.x[(i64)k * c.nc + parent_of(f.m, cf)];
  }
}

template <typename T>
void k_mg_prolong(int S, const LevelView<T>& coarse, const LevelView<T>& fine, Stream st) {
  launch(k_prolong_kernel<T>, nblk((i64)S * fine.nc), kT, 0, cs(st), S, coarse, fine);
}

// ------------------------------------------------------------------ coarsest grid
// One CTA: x = 0, `sweeps` red-black sweeps; for the space-time operator also
// the correction on the single aggregate of all cells (the Galerkin operator
// on the constant-per-slice space is the time-tridiagonal tau_G (2 d^k - d^{k-1} - d^{k+1}),
// tau_G = sum of tau over the cells), followed by `sweeps` more sweeps.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_kernel(int S, LevelView<T> L, int sweeps, T* lc, T* lr, T* agg) {
  i64 sq = (i64)L.m * L.m;
  i64 tot = (i64)S * L.nc;
  for (i64 i = threadIdx.x; i < tot; i += blockDim.x) L.x[i] = 0;
  __syncthreads();
  int passes = L.tau ? 2 : 1;
  for (int pass = 0; pass < passes; ++pass) {
    for (int it = 0; it < sweeps; ++it) {
      for (int color = 0; color < 2; ++color) {
        if (L.tau) {
          for (i64 i = threadIdx.x; i < sq; i += blockDim.x) line_gs(S, L, (i64)color * sq + i, lc, lr);
        } else {
          for (i64 i = threadIdx.x; i < (i64)S * sq; i += blockDim.x) {
            int k = (int)(i / sq);
            point_gs(S, L, k, (i64)color * sq + (i - (i64)k * sq));
          }
        }
        __syncthreads();
      }
    }
    if (!L.tau || pass == passes - 1) break;
    // aggregate correction
    for (i64 i = threadIdx.x; i < tot; i += blockDim.x) {
      int k = (int)(i / L.nc);
      L.r[i] = L.b[i] - level_apply(S, L, k, i - (i64)k * L.nc);
    }
    __syncthreads();
    // agg[0..S): rhs, agg[S..2S): tau_G, agg[2S..3S): cp, agg[3S..4S): solution
    for (int k = threadIdx.x; k < S; k += blockDim.x) {
      T rsum = 0, tsum = 0;
      for (i64 c = 0; c < L.nc; ++c) {
        rsum += L.r[(i64)k * L.nc + c];
        tsum += L.tau[(i64)k * L.nc + c];
      }
      agg[k] = rsum;
      agg[S + k] = tsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
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
    for (i64 i = threadIdx.x; i < tot; i += blockDim.x) L.x[i] += agg[3 * S + (int)(i / L.nc)];
    __syncthreads();
  }
}

template <typename T>
void k_mg_coarse_solve(int S, const LevelView<T>& L, int sweeps, T* line_c, T* line_r, T* agg, Stream st) {
  launch(k_coarse_kernel<T>, 1, 1024, 0, cs(st), S, L, sweeps, line_c, line_r, agg);
}

// ------------------------------------------------------------------ conversions
template <typename T>
__global__ void k_load_kernel(const double* src, double scale, T* b, T* x, i64 n) {
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
  GRID_LOOP(i, n) dst[i] = (double)x[i];
}
template <typename T>
void k_mg_store(const T* x, double* dst, i64 n, Stream st) {
  launch(k_store_kernel<T>, nblk(n), kT, 0, cs(st), x, dst, n);
}

#define OT_INST(T)                                                                                              \
  template void k_mg_lap_coef0<T>(const Dims&, const double*, const double*, const double*, T*, Stream);       \
  template void k_mg_schur_coef0<T>(const Dims&, const double*, const double*, T*, T*, Stream);                \
  template void k_mg_restrict_coef<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                  \
  template void k_mg_smooth<T>(int, const LevelView<T>&, int, T*, T*, Stream);                                 \
  template void k_mg_residual<T>(int, const LevelView<T>&, Stream);                                            \
  template void k_mg_restrict<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                       \
  template void k_mg_prolong<T>(int, const LevelView<T>&, const LevelView<T>&, Stream);                        \
  template void k_mg_coarse_solve<T>(int, const LevelView<T>&, int, T*, T*, T*, Stream);                       \
  template void k_mg_load<T>(const double*, double, T*, T*, i64, Stream);                                      \
  template void k_mg_store<T>(const T*, double*, i64, Stream);
OT_INST(float)
OT_INST(double)

}  // namespace ot

namespace ot {
template <typename T>
__global__ void k_axpy_t_kernel(const T* x, T a, T* y, i64 n) {
  GRID_LOOP(i, n) y[i] += a * x[i];
}
template <typename T>
void k_mg_axpy(const T* x, T a, T* y, i64 n, Stream st) {
  launch(k_axpy_t_kernel<T>, nblk(n), kT, 0, cs(st), x, a, y, n);
}
template void k_mg_axpy<float>(const float*, float, float*, i64, Stream);
template void k_mg_axpy<double>(const double*, double, double*, i64, Stream);
}  // namespace ot
