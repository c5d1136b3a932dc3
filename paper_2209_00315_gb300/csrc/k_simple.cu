// k_simple.cu -- the pieces of the SIMPLE preconditioner (Sec. 4.2) that the
// KKT kernels do not already provide: the diagonal of the potential block A,
// the time-line preconditioner of SIMPLE's Schur complement, and the
// element-wise scalings.  FP64 throughout.
//
// SIMPLE replaces A by A^ = Diag(A) in the block factorisation of the projected
// system [A, B^T P^T; P B, -P C P^T]; its Schur complement
//   S^ = -(P C P^T + P B A^-1 B^T P^T)
// couples coarse cell C of rho slice k with the same cell of slices k +- 1
// through the time differences J^T M (x^{k+1} - x^k)/dt of B, and with
// neighbouring cells through B's potential-gradient terms.  The inner solve of
// -S^ y = r is preconditioned by the time-line part L alone: per coarse cell C
// the tridiagonal matrix T_C over k = 0..K-1 with
//   diagonal     |C| s^k_C / rho^k_C + w^k_C + w^{k+1}_C,
//   off-diagonal -w^{k+1}_C between k and k+1,
//   w^j_C = sum over the four fine cells f of C of |f|^2 / (A^_{j,f} dt^2),
// which is all of -S^ when grad phi = 0.  The Krylov space lies in the range
// of P^T (zero slice sums), so the preconditioner solves P L P^T z = r there
// exactly: z = L^-1 (r - Y lambda) with Y the K slice indicators and
//   (Y^T L^-1 Y) lambda = Y^T L^-1 r,
// the K x K matrix G = Y^T L^-1 Y = sum_C T_C^-1 formed and Cholesky-factored
// once per Newton step with the line factors.
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

// Ad[jj N + c] = sum of the three edge weights of fine cell c in slice jj: the
// diagonal of A^{jj+1} = -div(rho~ grad) (boundary slots carry weight 0).
__global__ void k_simple_diag_kernel(Dims d, const double* __restrict__ kc, double* __restrict__ Ad) {
  OT_GRID_DEP_WAIT();
  const i64 n = (i64)(d.K + 1) * d.N;
  GRID_LOOP(i, n) {
    const i64 jj = i / d.N, c = i - jj * d.N;
    const double* w = kc + jj * 6 * d.N + c;
    Ad[i] = w[0] + w[d.N] + w[2 * d.N];
  }
}

// Time-line factors, one thread per coarse cell C: inv[k] = 1 / pivot_k and
// e[k] = the coupling of slices k and k+1 (e[K-1] unused), forward elimination
// of the tridiagonal system described above.
__global__ void k_simple_line_factor_kernel(Dims d, const double* __restrict__ kc, const double* __restrict__ Ad,
                                            double* __restrict__ inv, double* __restrict__ e) {
  OT_GRID_DEP_WAIT();
  const i64 C = blockIdx.x * (i64)blockDim.x + threadIdx.x;
  if (C >= d.Nc) return;
  i64 ch[4];
  children(d.n, decode(d.n, C), ch);
  const double f2 = d.area_f * d.area_f / (d.dt * d.dt);
  auto weight = [&](int j) {
    const double* a = Ad + (i64)j * d.N;
    return f2 * (1.0 / a[ch[0]] + 1.0 / a[ch[1]] + 1.0 / a[ch[2]] + 1.0 / a[ch[3]]);
  };
  const double* cdiag = kc + (i64)(d.K + 1) * 6 * d.N;  // |C| s/rho
  double w_lo = weight(0), w_hi = weight(1);
  double e_prev = 0.0, inv_prev = 0.0;
  for (int k = 0; k < d.K; ++k) {
    const i64 idx = (i64)k * d.Nc + C;
    const double diag = cdiag[idx] + w_lo + w_hi;
    const double piv = diag - e_prev * e_prev * inv_prev;
    const double ip = 1.0 / piv;
    const double ek = (k + 1 < d.K) ? -w_hi : 0.0;
    inv[idx] = ip;
    e[idx] = ek;
    e_prev = ek;
    inv_prev = ip;
    if (k + 1 < d.K) {
      w_lo = w_hi;
      w_hi = weight(k + 2);
    }
  }
}

// z = T^-1 (r - shift) per coarse cell (forward and back substitution over the
// K slices); shift[k] (nullable) is subtracted from every cell of slice k.  With
// r == nullptr the right-hand side is the indicator of slice `unit` instead.
// The forward pass stores u_k = y_k / pivot_k of the eliminated system.
__global__ void k_simple_line_solve_kernel(Dims d, const double* __restrict__ inv, const double* __restrict__ e,
                                           const double* __restrict__ r, const double* __restrict__ shift, int unit,
                                           double* __restrict__ z) {
  OT_GRID_DEP_WAIT();
  const i64 C = blockIdx.x * (i64)blockDim.x + threadIdx.x;
  if (C >= d.Nc) return;
  double prev = 0.0, e_prev = 0.0;
  for (int k = 0; k < d.K; ++k) {
    const i64 idx = (i64)k * d.Nc + C;
    double rk = r ? r[idx] : (k == unit ? 1.0 : 0.0);
    if (shift) rk -= shift[k];
    prev = (rk - e_prev * prev) * inv[idx];
    z[idx] = prev;
    e_prev = e[idx];
  }
  // back substitution: z_k = u_k - (e_k / pivot_k) z_{k+1}, from z_{K-1} = u_{K-1}
  double next = prev;
  for (int k = d.K - 2; k >= 0; --k) {
    const i64 idx = (i64)k * d.Nc + C;
    next = z[idx] - e[idx] * inv[idx] * next;
    z[idx] = next;
  }
}

// In-place Cholesky factor (lower, column-major, leading dimension K) of the
// K x K symmetric positive definite G by one CTA, left-looking by columns.
__global__ void k_simple_gram_factor_kernel(int K, double* G, int* status) {
  OT_GRID_DEP_WAIT();
  __shared__ double red[32];
  __shared__ double piv;
  for (int j = 0; j < K; ++j) {
    // pivot: G_jj - sum_{p<j} L_jp^2
    double a = 0.0;
    for (int p = threadIdx.x; p < j; p += blockDim.x) a += G[(i64)p * K + j] * G[(i64)p * K + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      const double dj = G[(i64)j * K + j] - t;
      if (!(dj > 0.0)) *status = 1;
      piv = dj > 0.0 ? sqrt(dj) : 1.0;
      G[(i64)j * K + j] = piv;
    }
    __syncthreads();
    // column below the pivot: L_ij = (G_ij - sum_{p<j} L_ip L_jp) / L_jj
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) {
      double v = G[(i64)j * K + i];
      for (int p = 0; p < j; ++p) v -= G[(i64)p * K + i] * G[(i64)p * K + j];
      G[(i64)j * K + i] = v / piv;
    }
    __syncthreads();
  }
}

// lambda = G^-1 t from the Cholesky factor (one CTA: forward then backward
// substitution, a column of updates per step).
__global__ void k_simple_gram_solve_kernel(int K, const double* __restrict__ L, const double* __restrict__ t,
                                           double* __restrict__ lam) {
  OT_GRID_DEP_WAIT();
  extern __shared__ double x[];
  for (int i = threadIdx.x; i < K; i += blockDim.x) x[i] = t[i];
  __syncthreads();
  for (int j = 0; j < K; ++j) {  // L y = t
    const double yj = x[j] / L[(i64)j * K + j];
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < K; i += blockDim.x) x[i] -= L[(i64)j * K + i] * yj;
    if (threadIdx.x == 0) x[j] = yj;
    __syncthreads();
  }
  for (int j = K - 1; j >= 0; --j) {  // L^T lambda = y
    const double lj = x[j] / L[(i64)j * K + j];
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += blockDim.x) x[i] -= L[(i64)i * K + j] * lj;
    if (threadIdx.x == 0) x[j] = lj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < K; i += blockDim.x) lam[i] = x[i];
}

// out = beta * out + alpha * num / den, element-wise.
__global__ void k_quot_kernel(const double* __restrict__ num, const double* __restrict__ den, double alpha,
                              double* __restrict__ out, double beta, i64 n) {
  OT_GRID_DEP_WAIT();
  GRID_LOOP(i, n) {
    const double q = alpha * num[i] / den[i];
    out[i] = (beta == 0.0) ? q : beta * out[i] + q;
  }
}

void k_simple_diag(const Dims& d, const double* kc, double* Ad, Stream st) {
  launch(k_simple_diag_kernel, nblk((i64)(d.K + 1) * d.N), kT, 0, cs(st), d, kc, Ad);
}

void k_simple_line_factor(const Dims& d, const double* kc, const double* Ad, double* inv, double* e, Stream st) {
  launch(k_simple_line_factor_kernel, nblk(d.Nc), kT, 0, cs(st), d, kc, Ad, inv, e);
}

void k_simple_line_solve(const Dims& d, const double* inv, const double* e, const double* r, const double* shift,
                         double* z, Stream st) {
  prof::begin(prof::SIMPLE_LINE, st);
  launch(k_simple_line_solve_kernel, nblk(d.Nc), kT, 0, cs(st), d, inv, e, r, shift, -1, z);
  // r, inv, e read; z written, then read and written back
  prof::end(prof::SIMPLE_LINE, st, 8.0 * 5.0 * (double)d.K * (double)d.Nc);
}

void k_simple_gram(const Dims& d, const double* inv, const double* e, double* scratch, double* G, int* status,
                   Stream st) {
  for (int k = 0; k < d.K; ++k) {
    launch(k_simple_line_solve_kernel, nblk(d.Nc), kT, 0, cs(st), d, inv, e, (const double*)nullptr,
           (const double*)nullptr, k, scratch);
    k_slice_sums(scratch, d.K, d.Nc, 1.0, G + (i64)k * d.K, st);  // column k: Y^T T^-1 e_k
  }
  launch(k_simple_gram_factor_kernel, 1, kT, 0, cs(st), d.K, G, status);
}

void k_simple_gram_solve(int K, const double* L, const double* t, double* lam, Stream st) {
  launch(k_simple_gram_solve_kernel, 1, kT, sizeof(double) * (size_t)K, cs(st), K, L, t, lam);
}

void k_quot(const double* num, const double* den, double alpha, double* out, double beta, i64 n, Stream st) {
  launch(k_quot_kernel, nblk(n), kT, 0, cs(st), num, den, alpha, out, beta, n);
}

}  // namespace ot
