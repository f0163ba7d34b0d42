// measure.h -- launcher of the Philox throughput kernel (model.cu) for api.cu; kept apart
// from internal.h so that the resampling kernels' sources do not depend on it.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace rsk {
cudaError_t launch_philox_throughput(int64_t threads, uint32_t draws_per_thread, uint64_t seed,
                                     uint32_t* xor_out, cudaStream_t st);
}  // namespace rsk
