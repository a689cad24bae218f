// Widening of the double-float intermediates (see intermediates.cuh).
#include <algorithm>

#include "cg_device.cuh"
#include "intermediates.cuh"

namespace enkf {

__global__ void df32_to_f64_kernel(const df32* __restrict__ src, double* __restrict__ dst, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < count; e += (int64_t)gridDim.x * kThreads)
    dst[e] = (double)src[e];
}

cudaError_t launch_df32_to_f64(const void* src, double* dst, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + kThreads - 1) / kThreads, 4096);
  df32_to_f64_kernel<<<blocks, kThreads, 0, s>>>(static_cast<const df32*>(src), dst, count);
  return cudaGetLastError();
}

}  // namespace enkf
