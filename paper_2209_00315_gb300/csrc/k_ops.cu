// k_ops.cu -- FP64 kernels of the discrete operators: residual F, the projected
// KKT operator, B^T, the BB Schur operator, cost/dual value and the pieces of
// the Newton update.  One thread per output entry; the bodies are in stencil.cuh.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "launch.cuh"
#include "ot_internal.h"

namespace ot {

static inline cudaStream_t cs(Stream s) { return reinterpret_cast<cudaStream_t>(s); }
static constexpr int kT = 256;
static constexpr int kRedBlocks = 608;

static inline int nblk(i64 n) {
  i64 b = (n + kT - 1) / kT;
  return (int)(b < 1 ? 1 : b);
}

#define GRID_LOOP(i, n) for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < (n); i += (i64)gridDim.x * blockDim.x)

__device__ __forceinline__ double warp_sum2(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ row-layout stencils
// A warp takes one row J of squares, its lanes the squares I (blockIdx.z walks
// the slices); each thread handles both triangles of its square.  Neighbours,
// parents and children by the row helpers of stencil.cuh; the operations are
// those of the per-cell bodies, in the same order.
static inline dim3 rows_grid(int side, int S) {
  return dim3((unsigned)((side + 31) / 32), (unsigned)((side + 7) / 8), (unsigned)(S < 65535 ? (S > 0 ? S : 1) : 65535));
}
static const dim3 kRowsBlock(32, 8);
#define ROWS_SQUARE(side, I, J)                    \
  const int I = blockIdx.x * 32 + threadIdx.x;     \
  const int J = blockIdx.y * 8 + threadIdx.y;      \
  if (I >= (side) || J >= (side)) return;

// u = M^{-1} B~ z (schur_u) on the fine grid.
template <typename T>
__global__ void __launch_bounds__(256) k_schur_u_rows(Dims d, const T* __restrict__ phi, const T* __restrict__ z,
                                                      T* __restrict__ u) {
  OT_GRID_DEP_WAIT();
  const int m = d.m, mm = m * m, N = (int)d.N, Nc = (int)d.Nc;
  ROWS_SQUARE(m, I, J)
  for (int jj = blockIdx.z; jj < d.K + 1; jj += gridDim.z) {
    const T* ph = phi + (i64)jj * N;
    const T* zm = (jj >= 1) ? z + (i64)(jj - 1) * Nc : nullptr;
    const T* zp = (jj <= d.K - 1) ? z + (i64)jj * Nc : nullptr;
    for (int t = 0; t < 2; ++t) {
      const int c = t * mm + J * m + I;
      const int P = row_parent(m, t, I, J);
      const T zmc = zm ? zm[P] : (T)0, zpc = zp ? zp[P] : (T)0;
      const T zbc = (T)0.5 * (zmc + zpc);
      const T pc = ph[c];
      T acc = (T)0;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        int Io, Jo;
        const int o = row_nb(m, t, I, J, sl, &Io, &Jo);
        if (o < 0) continue;
        const int Po = row_parent(m, 1 - t, Io, Jo);
        const T zbo = (T)0.5 * ((zm ? zm[Po] : (T)0) + (zp ? zp[Po] : (T)0));
        acc += (T)trans(sl) * (pc - ph[o]) * (zbc - zbo);
      }
      u[(i64)jj * N + c] = (zpc - zmc) / (T)d.dt + (T)0.5 * acc / (T)d.area_f;
    }
  }
}

// out = s (A~ z) - rho (B u) (schur_out) on the coarse grid.
template <typename T>
__global__ void __launch_bounds__(256) k_schur_out_rows(Dims d, const T* __restrict__ phi, const T* __restrict__ rho,
                                                        const T* __restrict__ s, const T* __restrict__ u,
                                                        const T* __restrict__ z, T* __restrict__ out) {
  OT_GRID_DEP_WAIT();
  const int n = d.n, nn = n * n, m = d.m, mm = m * m, N = (int)d.N, Nc = (int)d.Nc;
  ROWS_SQUARE(n, i, j)
  for (int k0 = blockIdx.z; k0 < d.K; k0 += gridDim.z) {
    const T* rk = rho + (i64)k0 * Nc;
    const T* zk = z + (i64)k0 * Nc;
    const T* p0 = phi + (i64)k0 * N;
    const T* p1 = p0 + N;
    const T* x0 = u + (i64)k0 * N;
    const T* x1 = x0 + N;
    for (int t = 0; t < 2; ++t) {
      const int C = t * nn + j * n + i;
      // A~ z (apply_atilde)
      T at = (T)0;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        int io, jo;
        const int O = row_nb(n, t, i, j, sl, &io, &jo);
        if (O < 0) continue;
        at += (T)trans(sl) * (T)0.5 * (rk[C] + rk[O]) * (zk[C] - zk[O]);
      }
      // B u (apply_B)
      int ct[4], cI[4], cJ[4];
      row_children(t, i, j, ct, cI, cJ);
      T acc = (T)0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int c = ct[a] * mm + cJ[a] * m + cI[a];
        acc += (T)d.area_f * (x1[c] - x0[c]) / (T)d.dt;
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
          int Io, Jo;
          const int o = row_nb(m, ct[a], cI[a], cJ[a], sl, &Io, &Jo);
          if (o < 0) continue;
          acc += (T)0.25 * (T)trans(sl) * ((p0[c] - p0[o]) * (x0[c] - x0[o]) + (p1[c] - p1[o]) * (x1[c] - x1[o]));
        }
      }
      const i64 idx = (i64)k0 * Nc + C;
      out[idx] = s[idx] * at - rho[idx] * acc;
    }
  }
}

// phi rows of [A, B^T P^T] x from the edge coefficients (kkt_phi_sliced).
// With e non-null (and with_a) it also writes e^jj_c = sum_slot g_slot (x_c - x_o), the
// B part of the rho rows at this cell, from the coefficients and values it has loaded.
__global__ void __launch_bounds__(256) k_kkt_phi_sliced_rows(Dims d, const double* __restrict__ kc,
                                                             const double* __restrict__ xp,
                                                             const double* __restrict__ yb, bool with_a,
                                                             double* __restrict__ y, double* __restrict__ e) {
  OT_GRID_DEP_WAIT();
  const int m = d.m, mm = m * m, N = (int)d.N, Nc = (int)d.Nc;
  ROWS_SQUARE(m, I, J)
  for (int jj = blockIdx.z; jj < d.K + 1; jj += gridDim.z) {
    const double* ybar = yb + (i64)jj * Nc;
    const double* ydif = yb + (i64)(d.K + 1 + jj) * Nc;
    const double* xs = with_a ? xp + (i64)jj * N : nullptr;
    for (int t = 0; t < 2; ++t) {
      const int c = t * mm + J * m + I;
      const int P = row_parent(m, t, I, J);
      double acc = ydif[P];
      const double ybc = ybar[P];
      const double xc = with_a ? xs[c] : 0.0;
      const double* kw = kc + (i64)jj * 6 * N + c;
      double ec = 0.0;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        int Io, Jo;
        const int o = row_nb(m, t, I, J, sl, &Io, &Jo);
        if (o < 0) continue;
        const double g = kw[(i64)(3 + sl) * N];
        acc += g * (ybc + ybar[row_parent(m, 1 - t, Io, Jo)]);
        if (with_a) {
          const double dx = xc - xs[o];
          acc += kw[(i64)sl * N] * dx;
          ec += g * dx;
        }
      }
      y[(i64)jj * N + c] = acc;
      if (e) e[(i64)jj * N + c] = ec;
    }
  }
}

// rho rows before the projection: (B x_phi)^k - |C| s/rho (x_rho - mean), the B part
// (apply_B_cached) summed over the four children from the edge sums e of the phi rows:
//   (B x)^k_C = sum_{c in C} [ |c| (x^{k+1}_c - x^k_c)/dt + (e^k_c + e^{k+1}_c)/2 ].
__global__ void __launch_bounds__(256) k_kkt_rho_rows(Dims d, const double* __restrict__ kc,
                                                      const double* __restrict__ xp, const double* __restrict__ e,
                                                      const double* __restrict__ xr,
                                                      const double* __restrict__ xmean, double* __restrict__ w) {
  OT_GRID_DEP_WAIT();
  const int n = d.n, nn = n * n, m = d.m, mm = m * m, N = (int)d.N, Nc = (int)d.Nc;
  const double* sr = kc + (i64)(d.K + 1) * 6 * d.N;
  ROWS_SQUARE(n, i, j)
  for (int k0 = blockIdx.z; k0 < d.K; k0 += gridDim.z) {
    const double* x0 = xp + (i64)k0 * N;
    const double* x1 = x0 + N;
    const double* e0 = e + (i64)k0 * N;
    const double* e1 = e0 + N;
    for (int t = 0; t < 2; ++t) {
      const int C = t * nn + j * n + i;
      int ct[4], cI[4], cJ[4];
      row_children(t, i, j, ct, cI, cJ);
      double dtime = 0.0, edges = 0.0;
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int c = ct[a] * mm + cJ[a] * m + cI[a];
        dtime += x1[c] - x0[c];
        edges += e0[c] + e1[c];
      }
      const i64 idx = (i64)k0 * Nc + C;
      w[idx] = d.af_dt * dtime + 0.5 * edges - sr[idx] * (xr[idx] - xmean[k0]);
    }
  }
}

// phi rows of [A, B^T P^T] x computed from phi (kkt_phi), for the FP32 B^T P^T of the preconditioner.
template <typename T>
__global__ void __launch_bounds__(256) k_kkt_phi_rows(Dims d, const T* __restrict__ phi, const T* __restrict__ rho,
                                                      const T* __restrict__ r0, const T* __restrict__ r1,
                                                      const T* __restrict__ xp, const T* __restrict__ xr,
                                                      const T* __restrict__ xmean, bool with_a, T* __restrict__ y) {
  OT_GRID_DEP_WAIT();
  const int m = d.m, mm = m * m, N = (int)d.N, Nc = (int)d.Nc;
  ROWS_SQUARE(m, I, J)
  for (int jj = blockIdx.z; jj < d.K + 1; jj += gridDim.z) {
    const T* ph = phi + (i64)jj * N;
    const T* xs = with_a ? xp + (i64)jj * N : nullptr;
    const T* ym = (jj >= 1) ? xr + (i64)(jj - 1) * Nc : nullptr;
    const T* yp = (jj <= d.K - 1) ? xr + (i64)jj * Nc : nullptr;
    const T mmn = (jj >= 1) ? xmean[jj - 1] : (T)0, mpn = (jj <= d.K - 1) ? xmean[jj] : (T)0;
    for (int t = 0; t < 2; ++t) {
      const int c = t * mm + J * m + I;
      const int P = row_parent(m, t, I, J);
      const T yma = ym ? ym[P] - mmn : (T)0, ypa = yp ? yp[P] - mpn : (T)0;
      T acc = (T)d.area_f * (yma - ypa) / (T)d.dt;
      const T ybc = (T)0.5 * (yma + ypa);
      const T rc = with_a ? rho_bar(d, rho, r0, r1, jj, (i64)P) : (T)0;
      const T pc = ph[c], xc = with_a ? xs[c] : (T)0;
#pragma unroll
      for (int sl = 0; sl < 3; ++sl) {
        int Io, Jo;
        const int o = row_nb(m, t, I, J, sl, &Io, &Jo);
        if (o < 0) continue;
        const int Po = row_parent(m, 1 - t, Io, Jo);
        const T ybo = (T)0.5 * ((ym ? ym[Po] - mmn : (T)0) + (yp ? yp[Po] - mpn : (T)0));
        T term = (T)0.5 * (ybc + ybo) * (pc - ph[o]);
        if (with_a) term += (T)0.5 * (rc + rho_bar(d, rho, r0, r1, jj, (i64)Po)) * (xc - xs[o]);
        acc += (T)trans(sl) * term;
      }
      y[(i64)jj * N + c] = acc;
    }
  }
}

// ------------------------------------------------------------------ residual
__global__ void k_residual_phi_kernel(Dims d, const double* phi, const double* rho, const double* r0,
                                      const double* r1, double* F) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(jj, d.K + 1, c, d.N) F[(i64)jj * d.N + c] = residual_phi(d, phi, rho, r0, r1, jj, c);
}

__global__ void k_residual_rho_kernel(Dims d, double mu, const double* phi, const double* rho, const double* s,
                                      double* Frho, double* Fs) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k0, d.K, C, d.Nc) {
    i64 i = (i64)k0 * d.Nc + C;
    Frho[i] = residual_rho(d, phi, s, k0, C);
    Fs[i] = rho[i] * s[i] - mu;
  }
}

void k_residual(const Dims& d, double mu, const double* phi, const double* rho, const double* s,
                const double* r0, const double* r1, double* Fphi, double* Frho, double* Fs, Stream st) {
  prof::begin(prof::RESIDUAL, st);
  launch(k_residual_phi_kernel, slice_grid(d.N, d.K + 1), kT, 0, cs(st), d, phi, rho, r0, r1, Fphi);
  launch(k_residual_rho_kernel, slice_grid(d.Nc, d.K), kT, 0, cs(st), d, mu, phi, rho, s, Frho, Fs);
  prof::end(prof::RESIDUAL, st, 8.0 * (2.0 * (d.K + 1) * d.N + 4.0 * d.K * d.Nc));
}

// ------------------------------------------------------------------ KKT operator
template <typename T>
__global__ void k_slice_mean_kernel(const T* x, i64 n, T* mean) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  const T* xs = x + (i64)blockIdx.x * n;
  double a = strided_sum(xs, n);
  a = warp_sum2(a);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
    mean[blockIdx.x] = (T)(t / (double)n);
  }
}

template <typename T>
__global__ void k_kkt_phi_kernel(Dims d, const T* phi, const T* rho, const T* r0, const T* r1, const T* xp,
                                 const T* xr, const T* xmean, bool with_a, T* y) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(jj, d.K + 1, c, d.N) y[(i64)jj * d.N + c] = kkt_phi(d, phi, rho, r0, r1, xp, xr, xmean, with_a, jj, c);
}

__global__ void k_kkt_rho_kernel(Dims d, const double* phi, const double* rho, const double* s, const double* xp,
                                 const double* xr, const double* xmean, double* w) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k0, d.K, C, d.Nc) w[(i64)k0 * d.Nc + C] = kkt_rho(d, phi, rho, s, xp, xr, xmean, k0, C);
}

// y_rho = w - slice mean(w) (P with equal coarse areas); wsum = slice sums of w.
__global__ void k_project_kernel(double* w, i64 n, double* wsum) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  __shared__ double mean;
  double* ws = w + (i64)blockIdx.x * n;
  double a = strided_sum(ws, n);
  a = warp_sum2(a);
  int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) sm[wp] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
    if (wsum) wsum[blockIdx.x] = t;
    mean = t / (double)n;
  }
  __syncthreads();
  for (i64 i = threadIdx.x; i < n; i += blockDim.x) ws[i] -= mean;
}

__global__ void k_kkt_coef_kernel(Dims d, const double* phi, const double* rho, const double* r0, const double* r1,
                                  double* kc) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(jj, d.K + 1, c, d.N) {
    double w[3], g[3];
    kkt_edge_coef(d, phi, rho, r0, r1, jj, c, w, g);
    double* o = kc + (i64)jj * 6 * d.N + c;
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) {
      o[(i64)sl * d.N] = w[sl];
      o[(i64)(3 + sl) * d.N] = g[sl];
    }
  }
}

__global__ void k_kkt_sr_kernel(Dims d, const double* rho, const double* s, double* sr) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, (i64)d.K * d.Nc) sr[i] = d.area_c * s[i] / rho[i];
}

void k_kkt_coef(const Dims& d, const double* phi, const double* rho, const double* s, const double* r0,
                const double* r1, double* kc, Stream st) {
  launch(k_kkt_coef_kernel, slice_grid(d.N, d.K + 1), kT, 0, cs(st), d, phi, rho, r0, r1, kc);
  launch(k_kkt_sr_kernel, nblk((i64)d.K * d.Nc), kT, 0, cs(st), d, rho, s, kc + (i64)(d.K + 1) * 6 * d.N);
}

// Slice values of the B^T part (kkt_slice_values) into the scratch of kc.
__global__ void k_kkt_slice_values_kernel(Dims d, const double* xr, const double* xmean, double* yb) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(jj, d.K + 1, C, d.Nc) kkt_slice_values(d, xr, xmean, jj, C, yb);
}



void k_kkt_apply(const Dims& d, const double* kc, const double* x, double* y, double* xmean, double* wsum,
                 Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N;
  const double* xr = x + Np;
  prof::begin(prof::KKT, st);
  double* yb = const_cast<double*>(kc) + kkt_yb_offset(d);
  launch(k_slice_mean_kernel<double>, d.K, 1024, 0, cs(st), xr, d.Nc, xmean);
  launch(k_kkt_slice_values_kernel, slice_grid(d.Nc, d.K + 1), kT, 0, cs(st), d, xr, (const double*)xmean, yb);
  double* e = const_cast<double*>(kc) + kkt_e_offset(d);
  launch(k_kkt_phi_sliced_rows, rows_grid(d.m, d.K + 1), kRowsBlock, 0, cs(st), d, kc, x, (const double*)yb, true, y,
         e);
  launch(k_kkt_rho_rows, rows_grid(d.n, d.K), kRowsBlock, 0, cs(st), d, kc, x, (const double*)e, xr,
         (const double*)xmean, y + Np);
  launch(k_project_kernel, d.K, 1024, 0, cs(st), y + Np, d.Nc, wsum);
  // x, y on both blocks, the six edge coefficients per fine cell and |C| s/rho
  prof::end(prof::KKT, st, 8.0 * (2.0 * Np + 2.0 * d.K * d.Nc + 6.0 * Np + d.K * d.Nc));
}

// ---- KKT operator with file-scope scratch (no allocation by the call).
// The slice means of x_rho live in this array instead of caller- or
// library-allocated memory; every GPU that loads the library holds it.
static __device__ __align__(256) double g_kkt_scratch[kStaticKktMaxK];
// Device address of the array per device, looked up once per device with that
// device current.  The lookup runs under a per-device once-flag, so two host
// threads making their first call on one device at the same time do not race.
static double* g_kkt_scratch_addr[kStaticKktMaxDevices];
static std::once_flag g_kkt_scratch_once[kStaticKktMaxDevices];

double* kkt_static_scratch() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) throw Error(7, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kStaticKktMaxDevices) throw Error(1, "device index beyond the static scratch table");
  // a failed lookup throws out of call_once, which leaves the flag unset: the next call retries
  std::call_once(g_kkt_scratch_once[dev], [dev]() {
    void* p = nullptr;
    const cudaError_t r = cudaGetSymbolAddress(&p, g_kkt_scratch);
    if (r != cudaSuccess) throw Error(7, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(r));
    g_kkt_scratch_addr[dev] = static_cast<double*>(p);
  });
  return g_kkt_scratch_addr[dev];
}

void k_kkt_apply_static(const Dims& d, const double* phi, const double* rho, const double* s, const double* r0,
                        const double* r1, const double* x, double* y, Stream st) {
  if (d.K > kStaticKktMaxK) throw Error(1, "K exceeds the static scratch of the no-allocation KKT operator");
  double* xmean = kkt_static_scratch();
  i64 Np = (i64)(d.K + 1) * d.N;
  const double* xr = x + Np;
  launch(k_slice_mean_kernel<double>, d.K, 1024, 0, cs(st), xr, d.Nc, xmean);
  launch(k_kkt_phi_kernel<double>, slice_grid(d.N, d.K + 1), kT, 0, cs(st), d, phi, rho, r0, r1, x, xr, xmean, true, y);
  launch(k_kkt_rho_kernel, slice_grid(d.Nc, d.K), kT, 0, cs(st), d, phi, rho, s, x, xr, xmean, y + Np);
  launch(k_project_kernel, d.K, 1024, 0, cs(st), y + Np, d.Nc, (double*)nullptr);
}

void k_bt_apply(const Dims& d, const double* kc, const double* yr, double* out_phi, double* yr_mean, Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N;
  prof::begin(prof::BT, st);
  launch(k_slice_mean_kernel<double>, d.K, 1024, 0, cs(st), yr, d.Nc, yr_mean);
  double* yb = const_cast<double*>(kc) + kkt_yb_offset(d);
  launch(k_kkt_slice_values_kernel, slice_grid(d.Nc, d.K + 1), kT, 0, cs(st), d, yr, (const double*)yr_mean, yb);
  launch(k_kkt_phi_sliced_rows, rows_grid(d.m, d.K + 1), kRowsBlock, 0, cs(st), d, kc, (const double*)nullptr,
         (const double*)yb, false, out_phi, (double*)nullptr);
  prof::end(prof::BT, st, 8.0 * (2.0 * Np + (double)d.K * d.Nc + 3.0 * Np));
}

// ------------------------------------------------------------------ Schur operator


void k_schur_apply(const Dims& d, const double* phi, const double* rho, const double* s, const double* z,
                   double* out, double* u, Stream st) {
  prof::begin(prof::SCHUR, st);
  launch(k_schur_u_rows<double>, rows_grid(d.m, d.K + 1), kRowsBlock, 0, cs(st), d, phi, z, u);
  launch(k_schur_out_rows<double>, rows_grid(d.n, d.K), kRowsBlock, 0, cs(st), d, phi, rho, s, (const double*)u, z,
         out);
  prof::end(prof::SCHUR, st, 8.0 * ((double)(d.K + 1) * d.N + 4.0 * d.K * d.Nc));
}

template <typename T>
__global__ void k_atilde_kernel(Dims d, const T* rho, const T* z, T* y) {
  OT_GRID_DEP_WAIT();
  SLICE_LOOP(k0, d.K, C, d.Nc) y[(i64)k0 * d.Nc + C] = apply_atilde(d, rho, z, k0, C) / (T)d.area_c;
}

void k_atilde_minv(const Dims& d, const double* rho, const double* z, double* y, Stream st) {
  launch(k_atilde_kernel<double>, slice_grid(d.Nc, d.K), kT, 0, cs(st), d, rho, z, y);
}

// ------------------------------------------------------------------ cost and dual value
__global__ void k_cost_dual_kernel(Dims d, const double* phi, const double* rho, const double* r0, const double* r1,
                                   double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sa[32], sb[32];
  i64 tot = (i64)(d.K + 1) * d.N;
  double a = 0.0, b = 0.0;
  GRID_LOOP(i, tot) {
    int jj = (int)(i / d.N);
    i64 c = i - (i64)jj * d.N;
    a += cost_cell(d, phi, rho, r0, r1, jj, c);
    if (jj == 0) b += dual_cell(d, phi, r0, r1, c);
  }
  a = warp_sum2(a);
  b = warp_sum2(b);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { ta += sa[q]; tb += sb[q]; }
    partial[2 * blockIdx.x] = ta;
    partial[2 * blockIdx.x + 1] = tb;
  }
}

__global__ void k_cost_dual_finish(const double* partial, int nb, double dt, double* out) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nb; ++q) { a += partial[2 * q]; b += partial[2 * q + 1]; }
  out[0] = dt * a;
  out[1] = b;
}

void k_cost_dual(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                 double* out, double* partial, Stream st) {
  launch(k_cost_dual_kernel, kRedBlocks, kT, 0, cs(st), d, phi, rho, r0, r1, partial);
  launch(k_cost_dual_finish, 1, 32, 0, cs(st), partial, kRedBlocks, d.dt, out);
}

// ------------------------------------------------------------------ Newton pieces
__global__ void k_newton_rhs_phi(const double* Fphi, double* f, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) f[i] = -Fphi[i];
}

// g~ = -F_rho - |c'| h / rho with h = -(F_s - mu); projected per slice, slice sums kept.
__global__ void k_newton_rhs_rho(Dims d, const double* Frho, const double* Fs, const double* rho, double* gt,
                                 double* hvec, double* gsum) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  __shared__ double mean;
  i64 base = (i64)blockIdx.x * d.Nc;
  double a = 0.0;
  for (i64 i = threadIdx.x; i < d.Nc; i += blockDim.x) {
    double h = -Fs[base + i];
    hvec[base + i] = h;
    double g = -Frho[base + i] - d.area_c * h / rho[base + i];
    gt[base + i] = g;
    a += g;
  }
  a = warp_sum2(a);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
    gsum[blockIdx.x] = t;
    mean = t / (double)d.Nc;
  }
  __syncthreads();
  for (i64 i = threadIdx.x; i < d.Nc; i += blockDim.x) gt[base + i] -= mean;
}

void k_newton_rhs(const Dims& d, const double* Fphi, const double* Frho, const double* Fs, const double* rho,
                  double* rhs, double* hvec, double* gsum, Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N;
  launch(k_newton_rhs_phi, nblk(Np), kT, 0, cs(st), Fphi, rhs, Np);
  launch(k_newton_rhs_rho, d.K, 512, 0, cs(st), d, Frho, Fs, rho, rhs + Np, hvec, gsum);
}

// ds = (h - s drho)/rho; candidate step min over negative directions of -x/dx, times tau.
__global__ void k_step_kernel(i64 n, const double* rho, const double* s, const double* drho, const double* h,
                              double* ds, double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  double a = INFINITY;
  GRID_LOOP(i, n) {
    double dsi = (h[i] - s[i] * drho[i]) / rho[i];
    ds[i] = dsi;
    if (drho[i] < 0.0) a = fmin(a, -rho[i] / drho[i]);
    if (dsi < 0.0) a = fmin(a, -s[i] / dsi);
  }
  for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_down_sync(0xffffffffu, a, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) a = fmin(a, sm[q]);
    partial[blockIdx.x] = a;
  }
}

__global__ void k_step_finish(const double* partial, int nb, double tau, double* out) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  double a = INFINITY;
  for (int q = 0; q < nb; ++q) a = fmin(a, partial[q]);
  out[0] = fmin(1.0, tau * a);
}

void k_step_length(const Dims& d, const double* rho, const double* s, const double* drho, const double* hvec,
                   double* ds, double tau, double* out, double* partial, Stream st) {
  i64 n = (i64)d.K * d.Nc;
  launch(k_step_kernel, kRedBlocks, kT, 0, cs(st), n, rho, s, drho, hvec, ds, partial);
  launch(k_step_finish, 1, 32, 0, cs(st), partial, kRedBlocks, tau, out);
}

__global__ void k_update_kernel(i64 Np, i64 Nr, const double* alpha_dev, double a_host, const double* dphi,
                                const double* drho, const double* ds, double* phi, double* rho, double* s) {
  OT_GRID_DEP_WAIT();
  double a = alpha_dev ? alpha_dev[0] : a_host;
  GRID_LOOP(i, Np) phi[i] += a * dphi[i];
  GRID_LOOP(i, Nr) {
    rho[i] += a * drho[i];
    s[i] += a * ds[i];
  }
}

void k_update(const Dims& d, const double* alpha_dev, double a_host, const double* dphi, const double* drho,
              const double* ds, double* phi, double* rho, double* s, Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N, Nr = (i64)d.K * d.Nc;
  launch(k_update_kernel, nblk(Np), kT, 0, cs(st), Np, Nr, alpha_dev, a_host, dphi, drho, ds, phi, rho, s);
}

__global__ void k_shift_const_kernel(int K, double dt, double area_total, const double* gsum, const double* wsum,
                                     double* cshift) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double c = 0.0;
  cshift[0] = 0.0;
  for (int k = 0; k < K; ++k) {
    c += dt * (gsum[k] - wsum[k]) / area_total;
    cshift[k + 1] = c;
  }
}

void k_shift_constants(const Dims& d, const double* gsum, const double* wsum, double area_total, double* cshift,
                       Stream st) {
  launch(k_shift_const_kernel, 1, 32, 0, cs(st), d.K, d.dt, area_total, gsum, wsum, cshift);
}

__global__ void k_rescale_kernel(Dims d, double* rho, const double* mass, double target) {
  OT_GRID_DEP_WAIT();
  i64 tot = (i64)d.K * d.Nc;
  GRID_LOOP(i, tot) rho[i] *= target / mass[i / d.Nc];
}

void k_rescale(const Dims& d, double* rho, const double* mass, double target, Stream st) {
  launch(k_rescale_kernel, nblk((i64)d.K * d.Nc), kT, 0, cs(st), d, rho, mass, target);
}

}  // namespace ot

namespace ot {
// Initial point (reading R8): rho^k = (1 - k dt) rho_in + k dt rho_f, phi = 0, s = mu0 / rho.
__global__ void k_init_point_kernel(Dims d, double mu0, const double* r0, const double* r1, double* phi,
                                    double* rho, double* s) {
  OT_GRID_DEP_WAIT();
  i64 Np = (i64)(d.K + 1) * d.N, Nr = (i64)d.K * d.Nc;
  GRID_LOOP(i, Np) phi[i] = 0.0;
  GRID_LOOP(i, Nr) {
    int k0 = (int)(i / d.Nc);
    i64 C = i - (i64)k0 * d.Nc;
    double t = (k0 + 1) * d.dt;
    double r = (1.0 - t) * r0[C] + t * r1[C];
    rho[i] = r;
    s[i] = mu0 / r;
  }
}

void k_init_point(const Dims& d, double mu0, const double* r0, const double* r1, double* phi, double* rho,
                  double* s, Stream st) {
  launch(k_init_point_kernel, nblk((i64)(d.K + 1) * d.N), kT, 0, cs(st), d, mu0, r0, r1, phi, rho, s);
}

// out = a .* b * scale
__global__ void k_mul_kernel(const double* a, const double* b, double scale, double* out, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) out[i] = scale * a[i] * b[i];
}
void k_mul(const double* a, const double* b, double scale, double* out, i64 n, Stream st) {
  launch(k_mul_kernel, nblk(n), kT, 0, cs(st), a, b, scale, out, n);
}

// Adjoint right-hand side dC/du: phi rows dt A^j phi^j, rho rows dt/4 R_T((grad phi^k)^2 + (grad phi^{k+1})^2),
// the rho rows projected (slice means removed, slice sums to gsum).
__global__ void k_adj_rhs_phi(Dims d, const double* phi, const double* rho, const double* r0, const double* r1,
                              double* out) {
  OT_GRID_DEP_WAIT();
  i64 tot = (i64)(d.K + 1) * d.N;
  GRID_LOOP(i, tot) {
    int jj = (int)(i / d.N);
    out[i] = d.dt * lap_apply(d, rho, r0, r1, phi, jj, i - (i64)jj * d.N);
  }
}

__global__ void k_adj_rhs_rho(Dims d, const double* phi, double* out) {
  OT_GRID_DEP_WAIT();
  i64 tot = (i64)d.K * d.Nc;
  GRID_LOOP(i, tot) {
    int k0 = (int)(i / d.Nc);
    i64 C = i - (i64)k0 * d.Nc;
    out[i] = d.dt * (kinetic_rho(d, phi, k0, C) + kinetic_rho(d, phi, k0 + 1, C));
  }
}

void k_adjoint_rhs(const Dims& d, const double* phi, const double* rho, const double* r0, const double* r1,
                   double* rhs, double* gsum, Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N;
  launch(k_adj_rhs_phi, nblk(Np), kT, 0, cs(st), d, phi, rho, r0, r1, rhs);
  launch(k_adj_rhs_rho, nblk((i64)d.K * d.Nc), kT, 0, cs(st), d, phi, rhs + Np);
  launch(k_project_kernel, d.K, 1024, 0, cs(st), rhs + Np, d.Nc, gsum);
}

// grad_in = dt/4 R_T (grad phi^1)^2 - lambda^T dF/drho_in, grad_f likewise with phi^{K+1}.
__global__ void k_adj_grad_kernel(Dims d, const double* phi, const double* lam, double* gin, double* gf) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(C, d.Nc) {
    gin[C] = d.dt * kinetic_rho(d, phi, 0, C) - adjoint_boundary(d, phi, lam, 0, 1.0, C);
    gf[C] = d.dt * kinetic_rho(d, phi, d.K, C) - adjoint_boundary(d, phi, lam, d.K, -1.0, C);
  }
}

void k_adjoint_grad(const Dims& d, const double* phi, const double* lam, double* gin, double* gf, Stream st) {
  launch(k_adj_grad_kernel, nblk(d.Nc), kT, 0, cs(st), d, phi, lam, gin, gf);
}
}  // namespace ot

namespace ot {
// ---- FP32 versions of the preconditioner's operators (mixed precision).
void k_bt_apply(const Dims& d, const float* phi, const float* yr, float* out_phi, float* yr_mean, Stream st) {
  i64 Np = (i64)(d.K + 1) * d.N;
  prof::begin(prof::BT, st);
  launch(k_slice_mean_kernel<float>, d.K, 1024, 0, cs(st), yr, d.Nc, yr_mean);
  launch(k_kkt_phi_rows<float>, rows_grid(d.m, d.K + 1), kRowsBlock, 0, cs(st), d, phi, (const float*)nullptr,
         (const float*)nullptr, (const float*)nullptr, (const float*)nullptr, yr, (const float*)yr_mean, false, out_phi);
  prof::end(prof::BT, st, 4.0 * (2.0 * Np + (double)d.K * d.Nc));
}

void k_schur_apply(const Dims& d, const float* phi, const float* rho, const float* s, const float* z, float* out,
                   float* u, Stream st) {
  prof::begin(prof::SCHUR, st);
  launch(k_schur_u_rows<float>, rows_grid(d.m, d.K + 1), kRowsBlock, 0, cs(st), d, phi, z, u);
  launch(k_schur_out_rows<float>, rows_grid(d.n, d.K), kRowsBlock, 0, cs(st), d, phi, rho, s, (const float*)u, z, out);
  prof::end(prof::SCHUR, st, 4.0 * ((double)(d.K + 1) * d.N + 4.0 * d.K * d.Nc));
}

void k_atilde_minv(const Dims& d, const float* rho, const float* z, float* y, Stream st) {
  launch(k_atilde_kernel<float>, slice_grid(d.Nc, d.K), kT, 0, cs(st), d, rho, z, y);
}

template <typename A, typename B>
__global__ void k_convert_kernel(const A* x, B* y, i64 n, double scale) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) y[i] = (B)(scale * (double)x[i]);
}
void k_convert(const double* x, float* y, i64 n, double scale, Stream st) {
  launch(k_convert_kernel<double, float>, nblk(n), kT, 0, cs(st), x, y, n, scale);
}
void k_convert(const float* x, double* y, i64 n, double scale, Stream st) {
  launch(k_convert_kernel<float, double>, nblk(n), kT, 0, cs(st), x, y, n, scale);
}

// out (float) = scale * a (float) .* b (double)
__global__ void k_mul_mixed_kernel(const float* a, const double* b, double scale, float* out, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) out[i] = (float)(scale * (double)a[i] * b[i]);
}
void k_mul(const float* a, const double* b, double scale, float* out, i64 n, Stream st) {
  launch(k_mul_mixed_kernel, nblk(n), kT, 0, cs(st), a, b, scale, out, n);
}

// y (float) = (float) c - y (the B^T P^T term), per element
__global__ void k_rsub_mixed_kernel(const double* c, float* y, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) y[i] = (float)c[i] - y[i];
}
void k_rsub(const double* c, float* y, i64 n, Stream st) { launch(k_rsub_mixed_kernel, nblk(n), kT, 0, cs(st), c, y, n); }
}  // namespace ot
