// k_krylov.cu -- device-controlled Arnoldi steps of the (F)GMRES solvers and
// the capture of their loops into CUDA graphs.
//
// Flexible GMRES (Sec. 3.1, the outer Krylov method of every Newton step) and
// the GMRES of the inner Schur solve (Sec. 4.3.3) keep their whole iteration
// state in device memory (kry::Ctl, the Hessenberg matrix, the Givens
// rotations and the rotated right-hand side g): the Gram-Schmidt passes read
// their vector count from the control block, one thread applies the Givens
// rotations and decides whether another step runs, and the least-squares
// solution and the update x += Z y need no host.  A loop of such steps is
// either enqueued eagerly (the host reads the status after each step) or
// captured once as a WHILE conditional node of a CUDA graph whose condition
// the Givens kernel sets; both run the same kernels in the same order.
#include <cuda_runtime.h>
#include <math.h>

#include <cstdio>
#include <vector>

#include "launch.cuh"
#include "ot_internal.h"

namespace ot {

static inline cudaStream_t cs(Stream s) { return reinterpret_cast<cudaStream_t>(s); }

static void cuda_ok(cudaError_t e, const char* where) {
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    throw Error(e == cudaErrorMemoryAllocation ? 8 : 7, buf);
  }
}

static constexpr int kDotBlocks = 608;  // 4 per SM, each walks one contiguous chunk of rows
static constexpr int kUpdBlocks = 608;  // 4 per SM
static constexpr int kThreads = 256;

// Layout of the scratch: per-block dot partials [kDotBlocks][mmax+2], then the
// update blocks' |w|^2 shares [kUpdBlocks], 64 spare, then 64 doubles holding
// the arrival counter of the update's last-block reduction (zeroed at
// allocation; each launch's last block resets it).
size_t kry_partial_doubles(int mmax) { return (size_t)kDotBlocks * (size_t)(mmax + 2) + kUpdBlocks + 128; }
size_t kry_counter_offset(int mmax) { return (size_t)kDotBlocks * (size_t)(mmax + 2) + kUpdBlocks + 64; }
static unsigned* upd_counter(double* partial, int mmax) {
  return reinterpret_cast<unsigned*>(partial + kry_counter_offset(mmax));
}

// True in the block that finishes last: every block publishes its global writes
// (fence), then counts itself in; the block that brings the count to gridDim.x
// sees every other block's partials and may reduce them (in a fixed order, so
// the result does not depend on which block came last).  That block resets the
// counter for the next launch.
__device__ __forceinline__ bool last_block_done(unsigned* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

template <typename T>
__device__ __forceinline__ T kwarp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double kwarp_sum(double v) { return kwarp_sum_t<double>(v); }

// 16-byte vectors of T: four floats or two doubles per load.
template <typename T>
struct Vec16;
template <>
struct Vec16<double> {
  typedef double2 type;
  static constexpr int E = 2;
  __device__ static double dot(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }
  __device__ static void unpack(const double2& v, double (&r)[2]) {
    r[0] = v.x;
    r[1] = v.y;
  }
  __device__ static double2 pack(const double (&r)[2]) { return make_double2(r[0], r[1]); }
};
template <>
struct Vec16<float> {
  typedef float4 type;
  static constexpr int E = 4;
  __device__ static float dot(const float4& a, const float4& b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
  __device__ static void unpack(const float4& v, float (&r)[4]) {
    r[0] = v.x;
    r[1] = v.y;
    r[2] = v.z;
    r[3] = v.w;
  }
  __device__ static float4 pack(const float (&r)[4]) { return make_float4(r[0], r[1], r[2], r[3]); }
};
template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  typedef double2 type;
};
template <>
struct Vec2<float> {
  typedef float2 type;
};

// Contiguous chunk [p0, p1) of np items for this block.
__device__ __forceinline__ void block_chunk(i64 np, i64* p0, i64* p1) {
  const i64 per = (np + gridDim.x - 1) / gridDim.x;
  *p0 = blockIdx.x * per;
  *p1 = min(np, *p0 + per);
}

// Rows of 16-byte loads: every basis row start and w on a 16-byte boundary.
static bool aligned16(const void* a, const void* b, i64 ld, size_t elem) {
  return (((uintptr_t)a | (uintptr_t)b) % 16) == 0 && ((size_t)ld * elem) % 16 == 0;
}

// ------------------------------------------------------------------ dot products
// partial[b * pstride + v] = this block's share of <V_v, w>, v < nv.  Warp w of
// the block takes vectors w, w + 8, ...; its lanes walk the block's chunk of
// rows with four 16-byte loads of V_v (and of w, an L1 hit after the first
// vector) in flight, sum in T and reduce across the warp in T (the cross-block
// sums are double).  No block barrier.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_kry_dot_kernel(const T* __restrict__ V, i64 ld,
                                                             const kry::Ctl* __restrict__ ctl, int add,
                                                             const T* __restrict__ w, i64 n, bool vec,
                                                             double* __restrict__ partial, int pstride) {
  OT_GRID_DEP_WAIT();
  typedef Vec16<T> VT;
  typedef typename VT::type V4;
  constexpr int E = VT::E;
  const int nv = ctl->j + add;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const i64 nq = vec ? n / E : 0;                  // 16-byte groups
  i64 q0, q1;
  block_chunk(nq, &q0, &q1);
  i64 e0 = nq * E, e1 = n;                         // scalar rows: the tail (or all rows when !vec)
  if (!vec) block_chunk(n, &e0, &e1);
  else if (blockIdx.x != gridDim.x - 1) e0 = e1;   // the vector tail belongs to the last block
  const V4* w4 = reinterpret_cast<const V4*>(w);
  for (int v = wp; v < nv; v += nw) {
    const T* xv = V + (i64)v * ld;
    const V4* x4 = reinterpret_cast<const V4*>(xv);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    i64 q = q0 + lane;
    for (; q + 96 < q1; q += 128) {
      const V4 x0 = x4[q], x1 = x4[q + 32], x2 = x4[q + 64], x3 = x4[q + 96];
      const V4 y0 = w4[q], y1 = w4[q + 32], y2 = w4[q + 64], y3 = w4[q + 96];
      a0 += VT::dot(x0, y0);
      a1 += VT::dot(x1, y1);
      a2 += VT::dot(x2, y2);
      a3 += VT::dot(x3, y3);
    }
    for (; q < q1; q += 32) a0 += VT::dot(x4[q], w4[q]);
    for (i64 i = e0 + lane; i < e1; i += 32) a1 += xv[i] * w[i];
    const T t = kwarp_sum_t<T>((a0 + a1) + (a2 + a3));
    if (lane == 0) partial[(i64)blockIdx.x * pstride + v] = (double)t;
  }
}

// out[v] = sum over blocks of partial[b * pstride + v], v < nv: one warp per v,
// fixed order, spread over many blocks (a single last block would walk the
// nv x blocks partials alone, which costs more than this launch).
__global__ void k_kry_dot_finish_kernel(const double* __restrict__ partial, int nb, int pstride,
                                        const kry::Ctl* __restrict__ ctl, int add, double* __restrict__ out) {
  OT_GRID_DEP_WAIT();
  const int nv = ctl->j + add;
  const int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= nv) return;
  double t = 0.0;
  for (int q = lane; q < nb; q += 32) t += partial[(i64)q * pstride + v];
  t = kwarp_sum(t);
  if (lane == 0) out[v] = t;
}

template <typename T>
void kry_dot(const T* V, i64 ld, const kry::Ctl* ctl, int add, int mmax, const T* w, i64 n, double* out,
             double* partial, int nv_hint, Stream s) {
  prof::begin(prof::MDOT, s);
  const int pstride = mmax + 2;
  launch(k_kry_dot_kernel<T>, kDotBlocks, kThreads, 0, cs(s), V, ld, ctl, add, w, n, aligned16(V, w, ld, sizeof(T)),
         partial, pstride);
  const int warps = kThreads / 32;
  launch(k_kry_dot_finish_kernel, (pstride + warps - 1) / warps, kThreads, 0, cs(s), (const double*)partial,
         kDotBlocks, pstride, ctl, add, out);
  // one pass over the nv basis vectors and w
  prof::end(prof::MDOT, s, nv_hint >= 0 ? (double)sizeof(T) * (nv_hint + 1.0) * (double)n : 0.0);
}

// ------------------------------------------------------------------ Givens step
// Column j of H: the two passes' coefficients, the norm after the second pass
// below the diagonal; the earlier rotations, then the one that zeroes H(j+1, j);
// the residual estimate, the status, j += 1 and the loop condition.  One thread.
__device__ void givens_step(const KryGivens& a) {
  kry::Ctl* c = a.ctl;
  const double* hc1 = a.hc1;
  const double* hc2 = a.hc2;
  const int j = c->j;
  double* col = a.H + (i64)j * a.ldh;
  const double hn = sqrt(fmax(hc2[j + 1], 0.0));
  double carry = (hc1 ? hc1[0] : 0.0) + hc2[0];
  for (int i = 0; i < j; ++i) {
    const double x = carry, y = (hc1 ? hc1[i + 1] : 0.0) + hc2[i + 1];
    col[i] = a.cs[i] * x + a.sn[i] * y;
    carry = -a.sn[i] * x + a.cs[i] * y;
  }
  const double x = carry, y = hn;
  const double den = hypot(x, y);
  const double cj = den > 0 ? x / den : 1.0, sj = den > 0 ? y / den : 0.0;
  a.cs[j] = cj;
  a.sn[j] = sj;
  col[j] = den;
  col[j + 1] = 0.0;
  const double gj = a.g[j];
  a.g[j + 1] = -sj * gj;
  a.g[j] = cj * gj;
  const double r = fabs(a.g[j + 1]);
  c->res = r;
  c->j = j + 1;
  c->total += 1;
  int st;
  if (!isfinite(r))
    st = kry::NONFINITE;
  else if (r <= c->tol)
    st = kry::CONVERGED;
  else if (hn <= 1e-14 * c->beta)
    st = kry::BREAKDOWN;
  else if (j + 1 >= c->m || c->base + j + 1 >= c->cap)
    st = kry::LIMIT;
  else
    st = kry::RUNNING;
  c->status = st;
  if (a.on) cudaGraphSetConditional((cudaGraphConditionalHandle)a.h, st == kry::RUNNING ? 1u : 0u);
}

// ------------------------------------------------------------------ update
// Block share of |w|^2 into partial[block] (after the block's rows are done);
// the last block then writes out[nv] = the sum of the shares (fixed order) and,
// when gv.ctl is set, takes the Givens step that consumes it.
__device__ __forceinline__ void block_norm_finish(double acc, double* partial, unsigned* counter, int nv,
                                                  double* out, const KryGivens& gv) {
  __shared__ double sm[kThreads / 32];
  const double a = kwarp_sum(acc);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sm[q];
    partial[blockIdx.x] = t;
  }
  if (!last_block_done(counter)) return;
  double t = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) t += __ldcg(partial + q);
  t = kwarp_sum(t);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot += sm[q];
    out[nv] = tot;
    if (gv.ctl) givens_step(gv);
    *counter = 0u;
  }
}

// w -= sum_{v < nv} h[v] V_v over the block's rows, in T; w32 (nullable) =
// float(new w); partial[block] = this block's share of |new w|^2 when norm is set.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_kry_update_kernel(const T* __restrict__ V, i64 ld,
                                                                const kry::Ctl* ctl, int add,
                                                                const double* __restrict__ h, T* w, i64 n,
                                                                bool vec, float* w32, double* norm_out,
                                                                double* __restrict__ partial, unsigned* counter,
                                                                KryGivens gv) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char kry_smem[];
  T* hs = reinterpret_cast<T*>(kry_smem);
  typedef Vec16<T> VT;
  typedef typename VT::type V4;
  constexpr int E = VT::E;
  const int nv = ctl->j + add;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) hs[v] = (T)h[v];
  __syncthreads();
  T acc = 0;
  const i64 nq = vec ? n / E : 0;
  i64 q0, q1;
  block_chunk(nq, &q0, &q1);
  i64 e0 = nq * E, e1 = n;
  if (!vec) block_chunk(n, &e0, &e1);
  else if (blockIdx.x != gridDim.x - 1) e0 = e1;
  V4* w4 = reinterpret_cast<V4*>(w);
  for (i64 q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    T r[E];
    VT::unpack(w4[q], r);
    int v = 0;
    for (; v + 8 <= nv; v += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        T x[E];
        VT::unpack(reinterpret_cast<const V4*>(V + (i64)(v + u) * ld)[q], x);
#pragma unroll
        for (int e = 0; e < E; ++e) r[e] -= hs[v + u] * x[e];
      }
    }
    for (; v < nv; ++v) {
      T x[E];
      VT::unpack(reinterpret_cast<const V4*>(V + (i64)v * ld)[q], x);
#pragma unroll
      for (int e = 0; e < E; ++e) r[e] -= hs[v] * x[e];
    }
    w4[q] = VT::pack(r);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (w32) w32[q * E + e] = (float)r[e];
      acc += r[e] * r[e];
    }
  }
  for (i64 i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
    T wi = w[i];
    for (int v = 0; v < nv; ++v) wi -= hs[v] * V[(i64)v * ld + i];
    w[i] = wi;
    if (w32) w32[i] = (float)wi;
    acc += wi * wi;
  }
  if (norm_out) block_norm_finish((double)acc, partial, counter, nv, norm_out, gv);
}

// The same update applied to an FP64 w from the FP32 copy of the basis, the
// combination sum_v h[v] V32_v formed in FP32: for the second Gram-Schmidt
// pass, whose coefficients are ~1e-7 of |w|, so that the FP32 rounding of the
// correction is ~1e-14 of |w| (FP64 level).  Reads 4 bytes per basis entry
// instead of 8 and keeps the FP64 units out of the loop.
__global__ void __launch_bounds__(kThreads) k_kry_update_shadow_kernel(const float* __restrict__ V, i64 ld,
                                                                       const kry::Ctl* ctl, int add,
                                                                       const double* __restrict__ h, double* w,
                                                                       i64 n, bool vec, double* norm_out,
                                                                       double* __restrict__ partial,
                                                                       unsigned* counter, KryGivens gv) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char kry_smem[];
  float* hs = reinterpret_cast<float*>(kry_smem);
  const int nv = ctl->j + add;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) hs[v] = (float)h[v];
  __syncthreads();
  double acc = 0.0;
  const i64 nq = vec ? n / 4 : 0;
  i64 q0, q1;
  block_chunk(nq, &q0, &q1);
  i64 e0 = nq * 4, e1 = n;
  if (!vec) block_chunk(n, &e0, &e1);
  else if (blockIdx.x != gridDim.x - 1) e0 = e1;
  for (i64 q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
    float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
    int v = 0;
    for (; v + 8 <= nv; v += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 x = reinterpret_cast<const float4*>(V + (i64)(v + u) * ld)[q];
        const float hv = hs[v + u];
        c.x += hv * x.x;
        c.y += hv * x.y;
        c.z += hv * x.z;
        c.w += hv * x.w;
      }
    }
    for (; v < nv; ++v) {
      const float4 x = reinterpret_cast<const float4*>(V + (i64)v * ld)[q];
      const float hv = hs[v];
      c.x += hv * x.x;
      c.y += hv * x.y;
      c.z += hv * x.z;
      c.w += hv * x.w;
    }
    double2* w2 = reinterpret_cast<double2*>(w) + 2 * q;
    double2 a = w2[0], b = w2[1];
    a.x -= (double)c.x;
    a.y -= (double)c.y;
    b.x -= (double)c.z;
    b.y -= (double)c.w;
    w2[0] = a;
    w2[1] = b;
    acc += a.x * a.x + a.y * a.y + b.x * b.x + b.y * b.y;
  }
  for (i64 i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
    float c = 0.f;
    for (int v = 0; v < nv; ++v) c += hs[v] * V[(i64)v * ld + i];
    const double wi = w[i] - (double)c;
    w[i] = wi;
    acc += wi * wi;
  }
  if (norm_out) block_norm_finish(acc, partial, counter, nv, norm_out, gv);
}


static KryGivens no_givens() {
  KryGivens g;
  g.ctl = nullptr;
  return g;
}

template <typename T>
void kry_update(const T* V, i64 ld, const kry::Ctl* ctl, int add, int mmax, const double* h, T* w, i64 n,
                float* w32, double* norm_out, double* partial, int nv_hint, Stream s, const KryGivens* gv) {
  prof::begin(prof::MUPDATE, s);
  const size_t smem = sizeof(T) * (size_t)(mmax + 2);
  const bool vec = aligned16(V, w, ld, sizeof(T));
  double* np = partial + (size_t)kDotBlocks * (size_t)(mmax + 2);
  launch(k_kry_update_kernel<T>, kUpdBlocks, kThreads, smem, cs(s), V, ld, ctl, add, h, w, n, vec, w32, norm_out,
         np, upd_counter(partial, mmax), (norm_out && gv) ? *gv : no_givens());
  // the nv basis vectors and w read, w (and its FP32 copy) written
  prof::end(prof::MUPDATE, s,
            nv_hint >= 0 ? (double)sizeof(T) * (nv_hint + 2.0) * (double)n + (w32 ? 4.0 * (double)n : 0.0) : 0.0);
}

void kry_update_shadow(const float* V32, i64 ld, const kry::Ctl* ctl, int add, int mmax, const double* h, double* w,
                       i64 n, double* norm_out, double* partial, int nv_hint, Stream s, const KryGivens* gv) {
  prof::begin(prof::MUPDATE, s);
  const size_t smem = sizeof(float) * (size_t)(mmax + 2);
  const bool vec = aligned16(V32, w, ld, sizeof(float)) && ((uintptr_t)w % 32) == 0;
  double* np = partial + (size_t)kDotBlocks * (size_t)(mmax + 2);
  launch(k_kry_update_shadow_kernel, kUpdBlocks, kThreads, smem, cs(s), V32, ld, ctl, add, h, w, n, vec, norm_out,
         np, upd_counter(partial, mmax), (norm_out && gv) ? *gv : no_givens());
  // the nv FP32 basis vectors read, w read and written
  prof::end(prof::MUPDATE, s, nv_hint >= 0 ? 4.0 * nv_hint * (double)n + 16.0 * (double)n : 0.0);
}

// ------------------------------------------------------------------ basis vectors
// With j = ctl->j + add: V_{j+1} = w / sqrt(nrm2[j+1]) (and its FP32 copy and
// `copy`), and Z_j = zsrc when zsrc is given.
template <typename T>
__global__ void k_kry_next_basis_kernel(const T* __restrict__ w, const double* __restrict__ nrm2,
                                        const kry::Ctl* __restrict__ ctl, int add, T* V, i64 ld, float* V32, T* copy,
                                        const T* __restrict__ zsrc, T* Z, i64 n) {
  OT_GRID_DEP_WAIT();
  const int j = ctl->j + add;
  const T f = (T)(1.0 / sqrt(nrm2[j + 1]));
  T* dst = V + (i64)(j + 1) * ld;
  float* d32 = V32 ? V32 + (i64)(j + 1) * ld : nullptr;
  T* zdst = zsrc ? Z + (i64)j * ld : nullptr;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T v = w[i] * f;
    dst[i] = v;
    if (d32) d32[i] = (float)v;
    if (copy) copy[i] = v;
    if (zdst) zdst[i] = zsrc[i];
  }
}

template <typename T>
void kry_next_basis(const T* w, const double* nrm2, const kry::Ctl* ctl, int add, T* V, i64 ld, float* V32, T* copy,
                    const T* zsrc, T* Z, i64 n, Stream s) {
  launch(k_kry_next_basis_kernel<T>, 1216, kThreads, 0, cs(s), w, nrm2, ctl, add, V, ld, V32, copy, zsrc, Z, n);
}

template <typename T>
__global__ void k_kry_start_basis_kernel(const T* __restrict__ r, const double* __restrict__ nrm2, T* V0, float* V32,
                                         T* copy, i64 n) {
  OT_GRID_DEP_WAIT();
  const T f = (T)(1.0 / sqrt(nrm2[0]));
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    const T v = r[i] * f;
    V0[i] = v;
    if (V32) V32[i] = (float)v;
    if (copy) copy[i] = v;
  }
}

template <typename T>
void kry_start_basis(const T* r, const double* nrm2, T* V0, float* V32_0, T* copy, i64 n, Stream s) {
  launch(k_kry_start_basis_kernel<T>, 1216, kThreads, 0, cs(s), r, nrm2, V0, V32_0, copy, n);
}

// ------------------------------------------------------------------ control
__global__ void k_kry_solve_init_kernel(kry::Ctl* c, const double* ref, int nref, double tol_rel, int cap) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  c->base = 0;
  c->cap = cap;
  if (nref > 0) {
    double t = 0.0;
    for (int i = 0; i < nref; ++i) t += ref[i];
    c->tol = tol_rel * sqrt(fmax(t, 0.0));
  }
}

void kry_solve_init(kry::Ctl* ctl, const double* ref, int nref, double tol_rel, int cap, Stream s) {
  launch(k_kry_solve_init_kernel, 1, 32, 0, cs(s), ctl, ref, nref, tol_rel, cap);
}

__global__ void k_kry_start_kernel(kry::Ctl* c, const double* nrm2, int m, double tol_rel, double* g,
                                   unsigned long long h, int on) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  const double beta = sqrt(fmax(nrm2[0], 0.0));
  c->beta = beta;
  c->j = 0;
  c->k = 0;
  c->m = m;
  if (tol_rel > 0.0) c->tol = tol_rel * beta;
  g[0] = beta;
  c->res = beta;
  int st;
  if (!isfinite(beta))
    st = kry::NONFINITE;
  else if (beta <= c->tol)
    st = kry::CONVERGED;
  else if (m <= 0 || c->base >= c->cap)
    st = kry::LIMIT;
  else
    st = kry::RUNNING;
  c->status = st;
  if (on) cudaGraphSetConditional((cudaGraphConditionalHandle)h, st == kry::RUNNING ? 1u : 0u);
}

void kry_start(kry::Ctl* ctl, const double* nrm2, int m, double tol_rel, double* g, CondHandle h, Stream s) {
  launch(k_kry_start_kernel, 1, 32, 0, cs(s), ctl, nrm2, m, tol_rel, g, h.h, (int)h.on);
}

// y = R^{-1} g[0..k) by columns (one warp): y_i = g_i / R_ii, then g_r -= R_ri y_i for r < i.
__global__ void k_kry_backsolve_kernel(kry::Ctl* __restrict__ c, const double* __restrict__ H, int ldh,
                                       const double* __restrict__ g, double* __restrict__ y) {
  OT_GRID_DEP_WAIT();
  extern __shared__ double gsm[];
  const int k = c->j;
  const int lane = threadIdx.x;
  for (int i = lane; i < k; i += 32) gsm[i] = g[i];
  for (int i = k - 1; i >= 0; --i) {
    __syncwarp();
    const double* col = H + (i64)i * ldh;
    const double d = col[i];
    const double v = d != 0.0 ? gsm[i] / d : 0.0;
    if (lane == 0) y[i] = v;
    for (int r = lane; r < i; r += 32) gsm[r] -= col[r] * v;
  }
  __syncwarp();
  if (lane == 0) {
    c->k = k;
    c->base += k;
  }
}

void kry_backsolve(kry::Ctl* ctl, const double* H, int ldh, const double* g, double* y, Stream s) {
  launch(k_kry_backsolve_kernel, 1, 32, sizeof(double) * (size_t)ldh, cs(s), ctl, H, ldh, g, y);
}

// x += sum_{v < k} y[v] Z_v over the block's rows.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_kry_combine_kernel(const T* __restrict__ Z, i64 ld,
                                                                 const kry::Ctl* __restrict__ ctl,
                                                                 const double* __restrict__ y, T* x, i64 n,
                                                                 bool pairs) {
  OT_GRID_DEP_WAIT();
  extern __shared__ __align__(16) unsigned char kry_smem[];
  T* ys = reinterpret_cast<T*>(kry_smem);
  const int nv = ctl->k;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) ys[v] = (T)y[v];
  __syncthreads();
  using V2 = typename Vec2<T>::type;
  if (pairs) {
    i64 p0, p1;
    block_chunk(n / 2, &p0, &p1);
    V2* x2 = reinterpret_cast<V2*>(x);
    for (i64 q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
      V2 a = x2[q];
      int v = 0;
      for (; v + 8 <= nv; v += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const V2 z = reinterpret_cast<const V2*>(Z + (i64)(v + u) * ld)[q];
          a.x += ys[v + u] * z.x;
          a.y += ys[v + u] * z.y;
        }
      }
      for (; v < nv; ++v) {
        const V2 z = reinterpret_cast<const V2*>(Z + (i64)v * ld)[q];
        a.x += ys[v] * z.x;
        a.y += ys[v] * z.y;
      }
      x2[q] = a;
    }
    if ((n & 1) && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
      T a = x[n - 1];
      for (int v = 0; v < nv; ++v) a += ys[v] * Z[(i64)v * ld + n - 1];
      x[n - 1] = a;
    }
  } else {
    i64 e0, e1;
    block_chunk(n, &e0, &e1);
    for (i64 i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
      T a = x[i];
      for (int v = 0; v < nv; ++v) a += ys[v] * Z[(i64)v * ld + i];
      x[i] = a;
    }
  }
}

template <typename T>
void kry_combine(const T* Z, i64 ld, const kry::Ctl* ctl, int mmax, const double* y, T* x, i64 n, int nv_hint,
                 Stream s) {
  prof::begin(prof::MCOMBINE, s);
  const bool pairs = (((uintptr_t)Z | (uintptr_t)x) % (2 * sizeof(T))) == 0 && (ld % 2) == 0;
  launch(k_kry_combine_kernel<T>, kUpdBlocks, kThreads, sizeof(T) * (size_t)(mmax + 2), cs(s), Z, ld, ctl, y, x, n,
         pairs);
  prof::end(prof::MCOMBINE, s, nv_hint >= 0 ? (double)sizeof(T) * (nv_hint + 2.0) * (double)n : 0.0);
}

#define OT_KRY_INST(T)                                                                                           \
  template void kry_dot<T>(const T*, i64, const kry::Ctl*, int, int, const T*, i64, double*, double*, int,     \
                           Stream);                                                                             \
  template void kry_update<T>(const T*, i64, const kry::Ctl*, int, int, const double*, T*, i64, float*,         \
                              double*, double*, int, Stream, const KryGivens*);                                 \
  template void kry_next_basis<T>(const T*, const double*, const kry::Ctl*, int, T*, i64, float*, T*, const T*, \
                                  T*, i64, Stream);                                                             \
  template void kry_start_basis<T>(const T*, const double*, T*, float*, T*, i64, Stream);                       \
  template void kry_combine<T>(const T*, i64, const kry::Ctl*, int, const double*, T*, i64, int, Stream);
OT_KRY_INST(double)
OT_KRY_INST(float)

// ------------------------------------------------------------------ loops and graphs
namespace dev {
namespace {
// Per thread: helper streams for capturing loop bodies (one per nesting
// depth), a pinned word for eager status reads, and the graph being captured.
thread_local std::vector<cudaStream_t> t_helpers;
thread_local int t_depth = 0;
thread_local kry::Ctl* t_ctl_host = nullptr;
struct LoopRec {
  const kry::Ctl* ctl;
  long long incl;      // launches captured in the body, nested loops' bodies included
  long long children;  // launches of the nested loops' bodies
  int parent;
};
thread_local std::vector<LoopRec>* t_loops = nullptr;  // loops of the graph being captured
thread_local int t_open = -1;                           // innermost loop being captured

cudaStream_t helper_stream(int depth) {
  while ((int)t_helpers.size() <= depth) {
    cudaStream_t s = nullptr;
    cuda_ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
    t_helpers.push_back(s);
  }
  return t_helpers[depth];
}
}  // namespace

bool capturing(Stream st) {
  cudaStreamCaptureStatus s = cudaStreamCaptureStatusNone;
  cuda_ok(cudaStreamIsCapturing(cs(st), &s), "cudaStreamIsCapturing");
  return s == cudaStreamCaptureStatusActive;
}

void read_ctl(const kry::Ctl* ctl, kry::Ctl* out, Stream st) {
  if (!t_ctl_host) {
    void* p = nullptr;
    cuda_ok(cudaMallocHost(&p, sizeof(kry::Ctl)), "cudaMallocHost");
    t_ctl_host = static_cast<kry::Ctl*>(p);
  }
  cuda_ok(cudaMemcpyAsync(t_ctl_host, ctl, sizeof(kry::Ctl), cudaMemcpyDeviceToHost, cs(st)), "cudaMemcpyAsync D2H");
  cuda_ok(cudaStreamSynchronize(cs(st)), "cudaStreamSynchronize");
  *out = *t_ctl_host;
}

long long device_while(Stream st, const kry::Ctl* ctl, const std::function<void(Stream, CondHandle)>& prologue,
                       const std::function<void(Stream, CondHandle, int)>& body) {
  if (!capturing(st)) {
    prologue(st, CondHandle{});
    long long per = 0;
    while (true) {
      kry::Ctl c;
      read_ctl(ctl, &c, st);
      if (c.status != kry::RUNNING) break;
      const long long a = prof::n_launch;
      body(st, CondHandle{}, c.j);
      per = prof::n_launch - a;
    }
    return per;
  }
  cudaStreamCaptureStatus cst;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cuda_ok(cudaStreamGetCaptureInfo(cs(st), &cst, nullptr, &g, &deps, nullptr, &nd), "cudaStreamGetCaptureInfo");
  cudaGraphConditionalHandle h;
  cuda_ok(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault), "cudaGraphConditionalHandleCreate");
  const CondHandle ch{(unsigned long long)h, true};
  prologue(st, ch);
  cuda_ok(cudaStreamGetCaptureInfo(cs(st), &cst, nullptr, &g, &deps, nullptr, &nd), "cudaStreamGetCaptureInfo");
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  cuda_ok(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p), "cudaGraphAddNode (while)");
  cuda_ok(cudaStreamUpdateCaptureDependencies(cs(st), &node, nullptr, 1, cudaStreamSetCaptureDependencies),
          "cudaStreamUpdateCaptureDependencies");
  cudaGraph_t bg = p.conditional.phGraph_out[0];
  cudaStream_t hs = helper_stream(t_depth);
  cuda_ok(cudaStreamBeginCaptureToGraph(hs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
          "cudaStreamBeginCaptureToGraph");
  int me = -1;
  if (t_loops) {
    t_loops->push_back(LoopRec{ctl, 0, 0, t_open});
    me = (int)t_loops->size() - 1;
  }
  const int saved_open = t_open;
  t_open = me;
  ++t_depth;
  const long long a = prof::t_captured;
  try {
    body((Stream)hs, ch, -1);
  } catch (...) {
    --t_depth;
    t_open = saved_open;
    cudaGraph_t dummy;
    cudaStreamEndCapture(hs, &dummy);
    throw;
  }
  const long long per = prof::t_captured - a;
  --t_depth;
  t_open = saved_open;
  cuda_ok(cudaStreamEndCapture(hs, &bg), "cudaStreamEndCapture (loop body)");
  if (me >= 0) {
    (*t_loops)[me].incl = per;
    if ((*t_loops)[me].parent >= 0) (*t_loops)[(*t_loops)[me].parent].children += per;
  }
  return per;
}

void Graph::capture(const std::function<void(Stream)>& enqueue) {
  release();
  cudaStream_t s = helper_stream(t_depth);
  std::vector<LoopRec> recs;
  t_loops = &recs;
  t_open = -1;
  ++t_depth;
  prof::capturing = true;
  const long long n0 = prof::t_captured;
  cudaGraph_t g = nullptr;
  auto cleanup = [&]() {
    prof::capturing = false;
    --t_depth;
    t_loops = nullptr;
    t_open = -1;
  };
  try {
    cuda_ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    try {
      enqueue((Stream)s);
    } catch (...) {
      cudaGraph_t dummy = nullptr;
      cudaStreamEndCapture(s, &dummy);
      if (dummy) cudaGraphDestroy(dummy);
      throw;
    }
    cuda_ok(cudaStreamEndCapture(s, &g), "cudaStreamEndCapture");
    cudaGraphExec_t ge = nullptr;
    cuda_ok(cudaGraphInstantiate(&ge, g, 0), "cudaGraphInstantiate");
    graph = g;
    exec = ge;
  } catch (...) {
    if (g) cudaGraphDestroy(g);
    cleanup();
    throw;
  }
  // captured launches are counted when the graph runs (Graph::executed)
  const long long captured = prof::t_captured - n0;
  long long in_loops = 0;
  loops.clear();
  for (const LoopRec& r : recs) {
    if (r.parent < 0) in_loops += r.incl;
    loops.push_back({r.ctl, r.incl - r.children});
  }
  static_launches = captured - in_loops;
  cleanup();
}

void Graph::launch(Stream st) {
  cuda_ok(cudaGraphLaunch((cudaGraphExec_t)exec, cs(st)), "cudaGraphLaunch");
}

long long Graph::executed(const std::vector<long long>& iterations) const {
  long long n = static_launches;
  for (size_t i = 0; i < loops.size() && i < iterations.size(); ++i) n += loops[i].second * iterations[i];
  return n;
}

void Graph::release() {
  if (exec) cudaGraphExecDestroy((cudaGraphExec_t)exec);
  if (graph) cudaGraphDestroy((cudaGraph_t)graph);
  exec = graph = nullptr;
  loops.clear();
  static_launches = 0;
}
}  // namespace dev

}  // namespace ot
