// Self-test of the failure detection: a wait that nothing ever releases must end at its time
// limit with the DS_TIMEOUT status bit, leaving the context usable. which = 0 runs the grid
// barrier of the persistent kernels with one CTA waiting for a second CTA that is not
// launched; which = 1 runs the bounded mbarrier wait of the tensor-core kernels on a barrier
// that no thread or MMA arrives on. Neither touches memory outside its own buffers.
#include "tc_mixed.cuh"

namespace enkf {

__global__ void selftest_wait_kernel(int which, unsigned long long timeout_ns, unsigned* buf) {
  __shared__ __align__(8) uint64_t mbar;
  int* status = reinterpret_cast<int*>(buf + 2);
  if (which == 0) {
    // a barrier over two CTAs entered by this one alone
    GridBarrier bar{buf, reinterpret_cast<int*>(buf + 1), status, 2u, 0u};
    bar.timeout_ns = timeout_ns;
    const bool ok = bar.sync();
    if (threadIdx.x == 0 && ok) buf[3] = 1u;   // released: must not happen
  } else {
    if (threadIdx.x == 0) mbar_init(&mbar);
    __syncthreads();
    const bool ok = mbar_wait(&mbar, 0u, status, timeout_ns);
    if (threadIdx.x == 0 && ok) buf[3] = 1u;
  }
}

cudaError_t selftest_wait_timeout(int which, double timeout_ms, cudaStream_t s, int* status_bits) {
  unsigned* buf = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    selftest_wait_kernel<<<1, 32, 0, s>>>(which, (unsigned long long)(timeout_ms * 1e6), buf);
    e = cudaGetLastError();
  }
  unsigned h[4] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(h, buf, sizeof(h), cudaMemcpyDeviceToHost);
  if (buf) cudaFree(buf);
  // status bits, plus bit 30 if the wait was released although nothing arrived
  if (status_bits) *status_bits = (int)h[2] | (h[3] ? (1 << 30) : 0);
  return e;
}

}  // namespace enkf
