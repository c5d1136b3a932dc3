// k_la.cu -- device memory helpers, reductions and BLAS-1 kernels (FP64).
//
// Reductions are deterministic: every block writes its partial result and a
// second one-block kernel adds the partials in a fixed order.
#include <cuda_runtime.h>
#include <math.h>

#include <chrono>
#include <cstdio>
#include <vector>

#include "launch.cuh"
#include "ot_internal.h"

namespace ot {

static inline cudaStream_t cs(Stream s) { return reinterpret_cast<cudaStream_t>(s); }

static void cuda_check(cudaError_t e, const char* where) {
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    throw Error(e == cudaErrorMemoryAllocation ? 8 : 7, buf);
  }
}

namespace prof {
bool enabled = false;
unsigned mask = 0;
std::atomic<long long> n_launch{0};
thread_local bool suspended = false;
thread_local bool capturing = false;
thread_local long long t_captured = 0;
int stride = 1;
namespace {
unsigned long long seen[COUNT] = {0};
struct Pending {
  int id;
  cudaEvent_t a, b;
  double bytes;
};
std::vector<cudaEvent_t> pool;
std::vector<Pending> pending;
std::vector<cudaEvent_t> open(COUNT, nullptr);
double ms_acc[COUNT] = {0};
long long n_acc[COUNT] = {0};
double b_acc[COUNT] = {0};
const char* names[COUNT] = {"kkt_apply", "gs_dot", "gs_update", "krylov_combine", "lap_smooth",
                            "schur_line_smooth", "mg_transfer", "schur_apply", "residual", "bt_apply",
                            "lap_lower_cycle", "schur_lower_cycle", "simple_line_solve"};
cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cuda_check(cudaEventCreate(&e), "cudaEventCreate");
  return e;
}
}  // namespace
void begin(int id, Stream s) {
  if (!enabled || suspended || capturing || !((mask >> id) & 1u)) return;
  if (++seen[id] % (unsigned long long)stride != 0) return;
  cudaEvent_t e = get_event();
  cudaEventRecord(e, cs(s));
  open[id] = e;
}
void end(int id, Stream s, double bytes) {
  if (!enabled || suspended || capturing || !open[id]) return;
  cudaEvent_t e = get_event();
  cudaEventRecord(e, cs(s));
  pending.push_back({id, open[id], e, bytes});
  open[id] = nullptr;
}
void harvest() {
  for (auto& p : pending) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    ms_acc[p.id] += ms;
    n_acc[p.id] += 1;
    b_acc[p.id] += p.bytes;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
}
void reset() {
  harvest();
  for (int i = 0; i < COUNT; ++i) ms_acc[i] = 0, n_acc[i] = 0, b_acc[i] = 0, seen[i] = 0;
}
const char* name(int id) { return (id >= 0 && id < COUNT) ? names[id] : ""; }
void read(int id, double* ms, long long* n, double* b) {
  harvest();
  *ms = ms_acc[id];
  *n = n_acc[id];
  *b = b_acc[id];
}
}  // namespace prof

namespace dev {
// Threads that drive their own stream allocate stream-ordered from the
// device's memory pool: no device-wide synchronisation on free, and freed
// blocks are reused by the next workspace.
thread_local bool pdl = false;
static thread_local cudaStream_t t_alloc_stream = nullptr;
void set_alloc_stream(Stream s) { t_alloc_stream = cs(s); }
static thread_local size_t t_krylov_budget = (size_t)64 << 30;
size_t krylov_budget() { return t_krylov_budget; }
void set_krylov_budget(size_t bytes) { t_krylov_budget = bytes; }

void* alloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = t_alloc_stream ? cudaMallocAsync(&p, bytes, t_alloc_stream) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof(buf), "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    throw Error(8, buf);
  }
  return p;
}
void release(void* p) {
  if (!p) return;
  if (t_alloc_stream)
    cudaFreeAsync(p, t_alloc_stream);
  else
    cudaFree(p);
}
void* host_alloc(size_t bytes) {
  void* p = nullptr;
  cuda_check(cudaMallocHost(&p, bytes ? bytes : 16), "cudaMallocHost");
  return p;
}
void host_release(void* p) {
  if (p) cudaFreeHost(p);
}
void copy_h2d(void* dst, const void* src, size_t bytes, Stream s) {
  cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs(s)), "cudaMemcpyAsync H2D");
}
void copy_d2h(void* dst, const void* src, size_t bytes, Stream s) {
  cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, cs(s)), "cudaMemcpyAsync D2H");
}
void copy_d2d(void* dst, const void* src, size_t bytes, Stream s) {
  cuda_check(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, cs(s)), "cudaMemcpyAsync D2D");
}
void zero(void* dst, size_t bytes, Stream s) { cuda_check(cudaMemsetAsync(dst, 0, bytes, cs(s)), "cudaMemsetAsync"); }
void sync(Stream s) {
  cuda_check(cudaStreamSynchronize(cs(s)), "cudaStreamSynchronize");
  if (prof::enabled && !prof::suspended) prof::harvest();
}
void check(const char* where) { cuda_check(cudaGetLastError(), where); }
bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
double now() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}
int current_device() {
  int d = 0;
  cuda_check(cudaGetDevice(&d), "cudaGetDevice");
  return d;
}
void set_device(int device) { cuda_check(cudaSetDevice(device), "cudaSetDevice"); }
Stream stream_create() {
  cudaStream_t s = nullptr;
  cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
  return (Stream)s;
}
void sync_quiet(Stream s) { cudaStreamSynchronize(cs(s)); }
void stream_destroy(Stream s) {
  if (!s) return;
  cudaStreamSynchronize(cs(s));
  cudaStreamDestroy(cs(s));
}
}  // namespace dev

// ------------------------------------------------------------------ helpers
static constexpr int kThreads = 256;
static constexpr int kRedBlocks = 608;  // 4 x 152 SMs

static inline int blocks_for(i64 n, int threads = kThreads, int cap = 1 << 20) {
  i64 b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

size_t k_reduce_scratch(int nv) { return (size_t)kRedBlocks * (nv + 1) + 64; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block; result valid in thread 0.  smem: blockDim/32 doubles.
// Two-element vector types for paired loads.
template <typename T>
struct Pair;
template <>
struct Pair<double> {
  typedef double2 type;
};
template <>
struct Pair<float> {
  typedef float2 type;
};

// Paired loads need every row start (base + v*ld) and w on a pair boundary.
template <typename T>
static bool pair_aligned(const T* V, i64 ld, const T* w) {
  const uintptr_t a = (uintptr_t)V | (uintptr_t)w;
  return (a % (2 * sizeof(T))) == 0 && (ld % 2) == 0;
}

__device__ __forceinline__ double block_sum(double v, double* smem) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// out[v] = sum_b partial[b * stride + v], v < nv (one block per v)
__global__ void k_finish_sum(const double* partial, int nblocks, int stride, int nv, double* out) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  int v = blockIdx.x;
  if (v >= nv) return;
  double a = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) a += partial[(i64)b * stride + v];
  a = block_sum(a, sm);
  if (threadIdx.x == 0) out[v] = a;
}

// ------------------------------------------------------------------ slice sums
template <typename T>
__global__ void k_slice_sums_kernel(const T* x, i64 n, double scale, T* sums) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  const T* xs = x + (i64)blockIdx.x * n;
  double a = strided_sum(xs, n);
  a = block_sum(a, sm);
  if (threadIdx.x == 0) sums[blockIdx.x] = (T)(scale * a);
}

void k_slice_sums(const double* x, int S, i64 n, double scale, double* sums, Stream s) {
  launch(k_slice_sums_kernel<double>, S, 1024, 0, cs(s), x, n, scale, sums);
}

template <typename T>
__global__ void k_slice_shift_kernel(T* x, int S, i64 n, const T* sums, double scale) {
  OT_GRID_DEP_WAIT();
  i64 tot = (i64)S * n;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < tot; i += (i64)gridDim.x * blockDim.x)
    x[i] -= (T)(scale * (double)sums[i / n]);
}

void k_slice_shift(double* x, int S, i64 n, const double* sums, double scale, Stream s) {
  i64 tot = (i64)S * n;
  launch(k_slice_shift_kernel<double>, blocks_for(tot, kThreads, 4096), kThreads, 0, cs(s), x, S, n, sums, scale);
}

// ------------------------------------------------------------------ Gram-Schmidt passes
// Dot products: blockIdx.y selects a group of 8 basis vectors, so a thread
// keeps 8 accumulators (high occupancy); w is re-read per group from L2.
template <typename T>
__global__ void __launch_bounds__(256) k_mdot8_kernel(const T* __restrict__ V, i64 ld, int nv,
                                                      const T* __restrict__ w, i64 n, bool pairs,
                                                      double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[8][8];
  const int v0 = blockIdx.y * 8;
  const int cnt = min(8, nv - v0);
  const T* Vg = V + (i64)v0 * ld;
  T acc[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) acc[v] = 0;
  // each block walks one contiguous chunk (few address-translation pages at a
  // time), two elements per load
  i64 done = 0;
  if (pairs) {
    using V2 = typename Pair<T>::type;
    const i64 np = n / 2, per = (np + gridDim.x - 1) / gridDim.x;
    const i64 p0 = blockIdx.x * per, p1 = min(np, p0 + per);
    const V2* w2 = reinterpret_cast<const V2*>(w);
    for (i64 q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
      const V2 wv = w2[q];
#pragma unroll
      for (int v = 0; v < 8; ++v)
        if (v < cnt) {
          const V2 x = reinterpret_cast<const V2*>(Vg + (i64)v * ld)[q];
          acc[v] += x.x * wv.x + x.y * wv.y;
        }
    }
    done = 2 * np;
  }
  for (i64 i = done + blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    T wi = w[i];
#pragma unroll
    for (int v = 0; v < 8; ++v)
      if (v < cnt) acc[v] += Vg[(i64)v * ld + i] * wi;
  }
  int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    double t = warp_sum((double)acc[v]);
    if (lane == 0) sm[v][wp] = t;
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sm[threadIdx.x][q];
    partial[(i64)blockIdx.x * (nv + 1) + v0 + threadIdx.x] = t;
  }
}

static int mdot_xblocks(int groups) {
  int bx = kRedBlocks / groups;
  return bx < 152 ? 152 : bx;
}

void k_mdot(const double* V, i64 ld, int nv, const double* w, i64 n, double* out, double* partial, Stream s) {
  prof::begin(prof::MDOT, s);
  int groups = (nv + 7) / 8;
  int bx = mdot_xblocks(groups);
  launch(k_mdot8_kernel<double>, dim3(bx, groups), 256, 0, cs(s), V, ld, nv, w, n, pair_aligned(V, ld, w),
         partial);
  launch(k_finish_sum, nv, 256, 0, cs(s), partial, bx, nv + 1, nv, out);
  prof::end(prof::MDOT, s, 8.0 * (double)(nv + 1) * (double)n);
}

// w -= sum_{v < nv} h[v] V_v (nv <= 64 per launch), streaming; optional squared
// norm of the new w into partial[block].
template <typename T>
__global__ void __launch_bounds__(256) k_update_kernel(const T* __restrict__ V, i64 ld, int nv,
                                                       const double* __restrict__ h, T* w, i64 n, bool pairs,
                                                       bool norm, double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ T hs[64];
  __shared__ double sm[32];
  for (int v = threadIdx.x; v < 64; v += blockDim.x) hs[v] = (v < nv) ? (T)h[v] : (T)0;
  __syncthreads();
  T acc = 0;
  i64 done = 0;
  if (pairs) {
    using V2 = typename Pair<T>::type;
    const i64 np = n / 2, per = (np + gridDim.x - 1) / gridDim.x;
    const i64 p0 = blockIdx.x * per, p1 = min(np, p0 + per);
    V2* w2 = reinterpret_cast<V2*>(w);
    for (i64 q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
      V2 wv = w2[q];
      int v = 0;
      for (; v + 8 <= nv; v += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const V2 x = reinterpret_cast<const V2*>(V + (i64)(v + u) * ld)[q];
          wv.x -= hs[v + u] * x.x;
          wv.y -= hs[v + u] * x.y;
        }
      }
      for (; v < nv; ++v) {
        const V2 x = reinterpret_cast<const V2*>(V + (i64)v * ld)[q];
        wv.x -= hs[v] * x.x;
        wv.y -= hs[v] * x.y;
      }
      w2[q] = wv;
      acc += wv.x * wv.x + wv.y * wv.y;
    }
    done = 2 * np;
  }
  for (i64 i = done + blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    T wi = w[i];
    int v = 0;
    for (; v + 8 <= nv; v += 8) {
#pragma unroll
      for (int u = 0; u < 8; ++u) wi -= hs[v + u] * V[(i64)(v + u) * ld + i];
    }
    for (; v < nv; ++v) wi -= hs[v] * V[(i64)v * ld + i];
    w[i] = wi;
    acc += wi * wi;
  }
  if (!norm) return;
  double a = block_sum((double)acc, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
}

void k_mupdate(const double* V, i64 ld, int nv, const double* h, double* w, i64 n, double* out, bool dots,
               bool norm, double* partial, Stream s) {
  prof::begin(prof::MUPDATE, s);
  for (int done = 0; done < nv; done += 64) {
    int c = nv - done < 64 ? nv - done : 64;
    bool last = done + c >= nv;
    launch(k_update_kernel<double>, kRedBlocks, 256, 0, cs(s), V + (i64)done * ld, ld, c, h + done, w, n,
           pair_aligned(V, ld, (const double*)w), norm && last, partial);
  }
  if (norm) launch(k_finish_sum, 1, 256, 0, cs(s), partial, kRedBlocks, 1, 1, out + nv);
  prof::end(prof::MUPDATE, s, 8.0 * (double)(nv + 2) * (double)n);
  if (dots) k_mdot(V, ld, nv, w, n, out, partial, s);
}

template <typename T>
__global__ void k_mcombine_kernel(const T* __restrict__ Z, i64 ld, int nv, const double* __restrict__ y, T* x,
                                  i64 n) {
  OT_GRID_DEP_WAIT();
  __shared__ T ys[64];
  for (int v = threadIdx.x; v < nv && v < 64; v += blockDim.x) ys[v] = (T)y[v];
  __syncthreads();
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    T a = x[i];
    for (int v = 0; v < nv; ++v) a += ys[v] * Z[(i64)v * ld + i];
    x[i] = a;
  }
}

void k_mcombine(const double* Z, i64 ld, int nv, const double* y, double* x, i64 n, Stream s) {
  prof::begin(prof::MCOMBINE, s);
  int done = 0;
  while (done < nv) {
    int c = nv - done;
    if (c > 64) c = 64;
    launch(k_mcombine_kernel<double>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), Z + (i64)done * ld, ld, c,
                                                                             y + done, x, n);
    done += c;
  }
  prof::end(prof::MCOMBINE, s, 8.0 * (double)(nv + 2) * (double)n);
}

template <typename T>
__global__ void k_dot_kernel(const T* x, const T* y, i64 n, double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  T t = 0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    t += x[i] * y[i];
  double a = block_sum((double)t, sm);
  if (threadIdx.x == 0) partial[blockIdx.x] = a;
}

void k_dot(const double* x, const double* y, i64 n, double* out, double* partial, Stream s) {
  launch(k_dot_kernel<double>, kRedBlocks, kThreads, 0, cs(s), x, y, n, partial);
  launch(k_finish_sum, 1, 256, 0, cs(s), partial, kRedBlocks, 1, 1, out);
}

__global__ void k_axpby_kernel(double a, const double* x, double b, double* y, i64 n) {
  OT_GRID_DEP_WAIT();
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
void k_axpby(double a, const double* x, double b, double* y, i64 n, Stream s) {
  launch(k_axpby_kernel, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), a, x, b, y, n);
}

template <typename T>
__global__ void k_scale_inv_norm_kernel(const T* x, const double* nrm2, T* y, i64 n) {
  OT_GRID_DEP_WAIT();
  T f = (T)(1.0 / sqrt(nrm2[0]));
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = x[i] * f;
}
void k_scale_by_inv_norm(const double* x, const double* nrm2, double* y, i64 n, Stream s) {
  launch(k_scale_inv_norm_kernel<double>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), x, nrm2, y, n);
}

template <typename T>
__global__ void k_scale_kernel(const T* x, T a, T* y, i64 n) {
  OT_GRID_DEP_WAIT();
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}
void k_scale(const double* x, double a, double* y, i64 n, Stream s) {
  launch(k_scale_kernel<double>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), x, a, y, n);
}
__global__ void k_fill_kernel(double* x, double v, i64 n) {
  OT_GRID_DEP_WAIT();
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) x[i] = v;
}
void k_fill(double* x, double v, i64 n, Stream s) {
  launch(k_fill_kernel, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), x, v, n);
}

// ------------------------------------------------------------------ max |x|, min x
__global__ void k_absmax_kernel(const double* x, i64 n, double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  __shared__ double sb[32];
  double a = 0.0, bad = 0.0;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x) {
    double v = x[i];
    if (!isfinite(v)) bad = 1.0;
    else a = fmax(a, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    bad = fmax(bad, __shfl_down_sync(0xffffffffu, bad, o));
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sm[w] = a; sb[w] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) { a = fmax(a, sm[q]); bad = fmax(bad, sb[q]); }
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = bad;
  }
}
__global__ void k_absmax_finish(const double* partial, int nb, double* out) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  double a = 0.0, bad = 0.0;
  for (int b = 0; b < nb; ++b) { a = fmax(a, partial[2 * b]); bad = fmax(bad, partial[2 * b + 1]); }
  out[0] = a;
  out[1] = bad;
}
void k_absmax(const double* x, i64 n, double* out, double* partial, Stream s) {
  launch(k_absmax_kernel, kRedBlocks, kThreads, 0, cs(s), x, n, partial);
  launch(k_absmax_finish, 1, 32, 0, cs(s), partial, kRedBlocks, out);
}

__global__ void k_min_kernel(const double* x, i64 n, double* partial) {
  OT_GRID_DEP_WAIT();
  __shared__ double sm[32];
  double a = INFINITY;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
    a = fmin(a, x[i]);
  for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_down_sync(0xffffffffu, a, o));
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sm[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) a = fmin(a, sm[q]);
    partial[blockIdx.x] = a;
  }
}
__global__ void k_min_finish(const double* partial, int nb, double* out) {
  OT_GRID_DEP_WAIT();
  if (threadIdx.x != 0) return;
  double a = INFINITY;
  for (int b = 0; b < nb; ++b) a = fmin(a, partial[b]);
  out[0] = a;
}
void k_min(const double* x, i64 n, double* out, double* partial, Stream s) {
  launch(k_min_kernel, kRedBlocks, kThreads, 0, cs(s), x, n, partial);
  launch(k_min_finish, 1, 32, 0, cs(s), partial, kRedBlocks, out);
}

}  // namespace ot

namespace ot {
// ---- FP32 vectors (the preconditioner's inner Krylov solve in mixed precision)
void k_slice_sums(const float* x, int S, i64 n, double scale, float* sums, Stream s) {
  launch(k_slice_sums_kernel<float>, S, 1024, 0, cs(s), x, n, scale, sums);
}
void k_slice_shift(float* x, int S, i64 n, const float* sums, double scale, Stream s) {
  i64 tot = (i64)S * n;
  launch(k_slice_shift_kernel<float>, blocks_for(tot, kThreads, 4096), kThreads, 0, cs(s), x, S, n, sums, scale);
}
void k_mdot(const float* V, i64 ld, int nv, const float* w, i64 n, double* out, double* partial, Stream s) {
  prof::begin(prof::MDOT, s);
  int groups = (nv + 7) / 8;
  int bx = mdot_xblocks(groups);
  launch(k_mdot8_kernel<float>, dim3(bx, groups), 256, 0, cs(s), V, ld, nv, w, n, pair_aligned(V, ld, w),
         partial);
  launch(k_finish_sum, nv, 256, 0, cs(s), partial, bx, nv + 1, nv, out);
  prof::end(prof::MDOT, s, 4.0 * (double)(nv + 1) * (double)n);
}
void k_mupdate(const float* V, i64 ld, int nv, const double* h, float* w, i64 n, double* out, bool dots, bool norm,
               double* partial, Stream s) {
  prof::begin(prof::MUPDATE, s);
  for (int done = 0; done < nv; done += 64) {
    int c = nv - done < 64 ? nv - done : 64;
    bool last = done + c >= nv;
    launch(k_update_kernel<float>, kRedBlocks, 256, 0, cs(s), V + (i64)done * ld, ld, c, h + done, w, n,
           pair_aligned(V, ld, (const float*)w), norm && last, partial);
  }
  if (norm) launch(k_finish_sum, 1, 256, 0, cs(s), partial, kRedBlocks, 1, 1, out + nv);
  prof::end(prof::MUPDATE, s, 4.0 * (double)(nv + 2) * (double)n);
  if (dots) k_mdot(V, ld, nv, w, n, out, partial, s);
}
void k_mcombine(const float* Z, i64 ld, int nv, const double* y, float* x, i64 n, Stream s) {
  prof::begin(prof::MCOMBINE, s);
  for (int done = 0; done < nv; done += 64) {
    int c = nv - done < 64 ? nv - done : 64;
    launch(k_mcombine_kernel<float>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), Z + (i64)done * ld, ld, c,
           y + done, x, n);
  }
  prof::end(prof::MCOMBINE, s, 4.0 * (double)(nv + 2) * (double)n);
}
void k_dot(const float* x, const float* y, i64 n, double* out, double* partial, Stream s) {
  launch(k_dot_kernel<float>, kRedBlocks, kThreads, 0, cs(s), x, y, n, partial);
  launch(k_finish_sum, 1, 256, 0, cs(s), partial, kRedBlocks, 1, 1, out);
}
void k_scale_by_inv_norm(const float* x, const double* nrm2, float* y, i64 n, Stream s) {
  launch(k_scale_inv_norm_kernel<float>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), x, nrm2, y, n);
}
void k_scale(const float* x, double a, float* y, i64 n, Stream s) {
  launch(k_scale_kernel<float>, blocks_for(n, kThreads, 4096), kThreads, 0, cs(s), x, (float)a, y, n);
}
}  // namespace ot
