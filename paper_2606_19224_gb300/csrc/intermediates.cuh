// Widening of the double-float arrays for enkf_copy_intermediates (the FP32 and tensor-core
// modes keep HA and the solution Z only as FP32 pairs).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace enkf {
// dst[e] = hi + lo of the double-float src[e], e < count, on stream s
cudaError_t launch_df32_to_f64(const void* src, double* dst, int64_t count, cudaStream_t s);
}  // namespace enkf
