// launch.cuh -- every kernel launch of the library goes through launch(), which
// counts it (prof::n_launch) before the <<<>>> launch on the given stream.
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

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  ++prof::n_launch;
  kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

}  // namespace ot
