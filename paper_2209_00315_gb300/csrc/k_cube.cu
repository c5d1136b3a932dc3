// k_cube.cu -- the discrete operators of the 3D Cartesian variant (the paper's
// test 4, Sec. 4.1): n^3 cubes of side h on [0,1]^3, density and potential on
// the same grid (J = I).  The TPFA formulas of Sec. 2.1 on this grid: every
// interior face has measure h^2 and joins two centres at distance h, so its
// transmissibility |e|/|w| is T = h, its weight W = |e||w| = h^3 and the edge
// reconstruction is the plain average (lambda = 1/2); every cell has volume
// V = h^3 and up to six face neighbours.  Cube (i, j, k) is cell (k n + j) n + i.
// The per-cell formulas are those of the triangle stencils with six face slots,
// unit transmissibility factor T, and the identity in place of parent/children.
#include <cuda_runtime.h>

#include "launch.cuh"
#include "ot_internal.h"

namespace ot {

static inline cudaStream_t cs(Stream s) { return reinterpret_cast<cudaStream_t>(s); }
static constexpr int kT = 256;

static inline int nblk(i64 n) {
  i64 b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : b);
}

#define GRID_LOOP(i, n) for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < (n); i += (i64)gridDim.x * blockDim.x)

CubeDims make_cube_dims(int n, int K) {
  CubeDims d;
  d.n = n;
  d.K = K;
  d.N = (i64)n * n * n;
  d.h = 1.0 / n;
  d.V = d.h * d.h * d.h;
  d.T = d.h;
  d.dt = 1.0 / (K + 1);
  return d;
}

// The face neighbours of cell c (-1 where the face is on the boundary).
__device__ __forceinline__ void cube_neighbours(const CubeDims& d, i64 c, i64 nb[6]) {
  const i64 n = d.n;
  const i64 i = c % n, j = (c / n) % n, k = c / (n * n);
  nb[0] = i > 0 ? c - 1 : -1;
  nb[1] = i < n - 1 ? c + 1 : -1;
  nb[2] = j > 0 ? c - n : -1;
  nb[3] = j < n - 1 ? c + n : -1;
  nb[4] = k > 0 ? c - n * n : -1;
  nb[5] = k < n - 1 ? c + n * n : -1;
}

// rho^k for k = 0..K+1 (paper index), the boundary data at both ends.
__device__ __forceinline__ double cube_rho_at(const CubeDims& d, const double* rho, const double* r0,
                                              const double* r1, int k, i64 c) {
  return k == 0 ? r0[c] : (k == d.K + 1 ? r1[c] : rho[(i64)(k - 1) * d.N + c]);
}

// Mean density of potential slice jj: (rho^jj + rho^{jj+1}) / 2.
__device__ __forceinline__ double cube_rho_bar(const CubeDims& d, const double* rho, const double* r0,
                                               const double* r1, int jj, i64 c) {
  return 0.5 * (cube_rho_at(d, rho, r0, r1, jj, c) + cube_rho_at(d, rho, r0, r1, jj + 1, c));
}

// F_phi (K+1 slices), F_rho and F_s - mu (K slices) of Eq. conservation_discrete,
// hj_discrete (time term J^T M, reading R3) and ortho_discrete.
__global__ void k_cube_residual_phi_kernel(CubeDims d, const double* phi, const double* rho, const double* r0,
                                           const double* r1, double* F) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(idx, (i64)(d.K + 1) * d.N) {
    const int jj = (int)(idx / d.N);
    const i64 c = idx - (i64)jj * d.N;
    const double* ph = phi + (i64)jj * d.N;
    const double ra = cube_rho_at(d, rho, r0, r1, jj, c), rb = cube_rho_at(d, rho, r0, r1, jj + 1, c);
    const double rc = 0.5 * (ra + rb);
    double acc = -d.V * (rb - ra) / d.dt;
    i64 nb[6];
    cube_neighbours(d, c, nb);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (nb[f] < 0) continue;
      acc += d.T * 0.5 * (rc + cube_rho_bar(d, rho, r0, r1, jj, nb[f])) * (ph[c] - ph[nb[f]]);
    }
    F[idx] = acc;
  }
}

__global__ void k_cube_residual_rho_kernel(CubeDims d, double mu, const double* phi, const double* rho,
                                           const double* s, double* Frho, double* Fs) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(idx, (i64)d.K * d.N) {
    const int k0 = (int)(idx / d.N);
    const i64 c = idx - (i64)k0 * d.N;
    const double* p0 = phi + (i64)k0 * d.N;
    const double* p1 = p0 + d.N;
    double acc = d.V * (p1[c] - p0[c]) / d.dt + d.V * s[idx];
    i64 nb[6];
    cube_neighbours(d, c, nb);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      if (nb[f] < 0) continue;
      const double g0 = p0[c] - p0[nb[f]], g1 = p1[c] - p1[nb[f]];
      acc += 0.125 * d.T * (g0 * g0 + g1 * g1);
    }
    Frho[idx] = acc;
    Fs[idx] = rho[idx] * s[idx] - mu;
  }
}

// Potential rows of the projected KKT operator [A, B^T P^T; P B, -P C P^T]
// (Eq. newton-linsys-shift-reduced-projected) on x = (x_phi; x_rho), y = P^T x_rho
// (slice means ymean removed): A x_phi + B^T y.
__global__ void k_cube_kkt_phi_kernel(CubeDims d, const double* phi, const double* rho, const double* r0,
                                      const double* r1, const double* x, const double* ymean, double* out) {
  OT_GRID_DEP_WAIT();
  const i64 Np = (i64)(d.K + 1) * d.N;
  const double* xr = x + Np;
  GRID_LOOP(idx, Np) {
    const int jj = (int)(idx / d.N);
    const i64 c = idx - (i64)jj * d.N;
    const double* ph = phi + (i64)jj * d.N;
    const double* xs = x + (i64)jj * d.N;
    auto y_at = [&](int k0, i64 cell) {  // P^T x_rho on rho slice k0 (0 outside 0..K-1)
      return (k0 >= 0 && k0 < d.K) ? xr[(i64)k0 * d.N + cell] - ymean[k0] : 0.0;
    };
    const double ym = y_at(jj - 1, c), yp = y_at(jj, c);
    double acc = d.V * (ym - yp) / d.dt;
    const double ybc = 0.5 * (ym + yp), rc = cube_rho_bar(d, rho, r0, r1, jj, c);
    i64 nb[6];
    cube_neighbours(d, c, nb);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const i64 o = nb[f];
      if (o < 0) continue;
      const double ybo = 0.5 * (y_at(jj - 1, o) + y_at(jj, o));
      acc += d.T * (0.5 * (ybc + ybo) * (ph[c] - ph[o]) +
                    0.5 * (rc + cube_rho_bar(d, rho, r0, r1, jj, o)) * (xs[c] - xs[o]));
    }
    out[idx] = acc;
  }
}

// Density rows before the projection: w = B x_phi - C P^T x_rho, C = M' diag(s/rho).
__global__ void k_cube_kkt_rho_kernel(CubeDims d, const double* phi, const double* rho, const double* s,
                                      const double* x, const double* ymean, double* w) {
  OT_GRID_DEP_WAIT();
  const i64 Np = (i64)(d.K + 1) * d.N;
  GRID_LOOP(idx, (i64)d.K * d.N) {
    const int k0 = (int)(idx / d.N);
    const i64 c = idx - (i64)k0 * d.N;
    const double* p0 = phi + (i64)k0 * d.N;
    const double* p1 = p0 + d.N;
    const double* x0 = x + (i64)k0 * d.N;
    const double* x1 = x0 + d.N;
    double acc = d.V * (x1[c] - x0[c]) / d.dt;
    i64 nb[6];
    cube_neighbours(d, c, nb);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const i64 o = nb[f];
      if (o < 0) continue;
      acc += 0.25 * d.T * ((p0[c] - p0[o]) * (x0[c] - x0[o]) + (p1[c] - p1[o]) * (x1[c] - x1[o]));
    }
    w[idx] = acc - d.V * s[idx] / rho[idx] * (x[Np + idx] - ymean[k0]);
  }
}

// Per-cell shares of the cost C and the dual value D (reading R15); each face
// is seen from both of its cells, hence the halves.
__global__ void k_cube_cost_dual_kernel(CubeDims d, const double* phi, const double* rho, const double* r0,
                                        const double* r1, double* cc, double* dc) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(c, d.N) {
    i64 nb[6];
    cube_neighbours(d, c, nb);
    double cost = 0.0;
    for (int jj = 0; jj <= d.K; ++jj) {
      const double* ph = phi + (i64)jj * d.N;
      const double rc = cube_rho_bar(d, rho, r0, r1, jj, c);
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        if (nb[f] < 0) continue;
        const double g = ph[c] - ph[nb[f]];
        cost += 0.25 * d.T * 0.5 * (rc + cube_rho_bar(d, rho, r0, r1, jj, nb[f])) * g * g;
      }
    }
    cc[c] = d.dt * cost;
    const double* pf = phi;
    const double* pl = phi + (i64)d.K * d.N;
    double corr = 0.0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const i64 o = nb[f];
      if (o < 0) continue;
      const double g1 = pf[c] - pf[o], gK = pl[c] - pl[o];
      corr += 0.5 * d.T * (0.5 * (r0[c] + r0[o]) * g1 * g1 + 0.5 * (r1[c] + r1[o]) * gK * gK);
    }
    dc[c] = d.V * (pl[c] * r1[c] - pf[c] * r0[c]) - 0.25 * d.dt * corr;
  }
}

void k_cube_residual(const CubeDims& d, double mu, const double* phi, const double* rho, const double* s,
                     const double* r0, const double* r1, double* Fphi, double* Frho, double* Fs, Stream st) {
  launch(k_cube_residual_phi_kernel, nblk((i64)(d.K + 1) * d.N), kT, 0, cs(st), d, phi, rho, r0, r1, Fphi);
  launch(k_cube_residual_rho_kernel, nblk((i64)d.K * d.N), kT, 0, cs(st), d, mu, phi, rho, s, Frho, Fs);
}

void k_cube_kkt_apply(const CubeDims& d, const double* phi, const double* rho, const double* s, const double* r0,
                      const double* r1, const double* x, double* y, double* scratch, Stream st) {
  const i64 Np = (i64)(d.K + 1) * d.N;
  double* ymean = scratch;
  double* wmean = scratch + d.K;
  k_slice_sums(x + Np, d.K, d.N, 1.0 / (double)d.N, ymean, st);
  launch(k_cube_kkt_phi_kernel, nblk(Np), kT, 0, cs(st), d, phi, rho, r0, r1, x, (const double*)ymean, y);
  launch(k_cube_kkt_rho_kernel, nblk((i64)d.K * d.N), kT, 0, cs(st), d, phi, rho, s, x, (const double*)ymean,
         y + Np);
  // P: remove each slice's mean (uniform cells)
  k_slice_sums(y + Np, d.K, d.N, 1.0 / (double)d.N, wmean, st);
  k_slice_shift(y + Np, d.K, d.N, wmean, 1.0, st);
}

void k_cube_cost_dual(const CubeDims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                      double* out, double* scratch, Stream st) {
  double* cc = scratch;
  double* dc = scratch + d.N;
  launch(k_cube_cost_dual_kernel, nblk(d.N), kT, 0, cs(st), d, phi, rho, r0, r1, cc, dc);
  k_slice_sums(cc, 2, d.N, 1.0, out, st);   // out[0] = C, out[1] = D
}

}  // namespace ot
