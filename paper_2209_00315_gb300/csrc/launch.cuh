// launch.cuh -- every kernel launch of the library goes through launch(), which
// counts it (prof::n_launch) before the <<<>>> launch on the given stream.
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "ot_internal.h"

namespace ot {

template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  ++prof::n_launch;
  kernel<<<grid, block, smem, st>>>(std::forward<Args>(args)...);
}

}  // namespace ot
