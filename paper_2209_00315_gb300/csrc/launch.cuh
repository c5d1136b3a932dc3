// launch.cuh -- every kernel launch of the library goes through launch(), which
// counts it (prof::n_launch; into a graph: prof::t_captured) and launches it on
// the given stream (with programmatic dependent launch when dev::pdl is set).
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "ot_internal.h"

namespace ot {

// Grid for S slices of n cells each: blockIdx.y walks the slices (no division
// to split a flat index), blockIdx.x / threadIdx.x the cells of a slice.
inline dim3 slice_grid(long long n, int S, int threads = 256) {
  long long bx = (n + threads - 1) / threads;
  if (bx < 1) bx = 1;
  return dim3((unsigned)bx, (unsigned)(S < 65535 ? (S > 0 ? S : 1) : 65535), 1);
}

#define SLICE_LOOP(k, S, c, n)                                          \
  for (int k = blockIdx.y; k < (S); k += gridDim.y)                     \
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; \
         c < (n); c += (long long)gridDim.x * blockDim.x)

// This thread's share of sum_i xs[i] over a strided walk of n values, in
// double, with four independent loads in flight per iteration: a block
// reduces one slice of tens of thousands of values, and a single dependent
// accumulator would wait for each load in turn.
// The per-thread partial sums are in T: a block of one slice runs on one SM,
// where FP64 adds of FP32 data would cost more than the loads.
template <typename T>
__device__ __forceinline__ double strided_sum(const T* xs, long long n) {
  const long long b = blockDim.x;
  T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  long long i = threadIdx.x;
  for (; i + 3 * b < n; i += 4 * b) {
    a0 += xs[i];
    a1 += xs[i + b];
    a2 += xs[i + 2 * b];
    a3 += xs[i + 3 * b];
  }
  for (; i < n; i += b) a0 += xs[i];
  return (double)((a0 + a1) + (a2 + a3));
}

// First statement of every kernel: wait until the grid this launch depends on
// has completed and its writes are visible (a no-op for a launch without the
// programmatic-serialisation attribute).
#define OT_GRID_DEP_WAIT() asm volatile("griddepcontrol.wait;" ::: "memory")

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  if (prof::capturing)
    ++prof::t_captured;  // counted when the graph runs
  else
    ++prof::n_launch;
  if (dev::pdl) {
    // programmatic dependent launch: the grid may be scheduled while its predecessor's last
    // blocks run; the kernel's OT_GRID_DEP_WAIT keeps the data dependency
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    return;
  }
  kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

}  // namespace ot
