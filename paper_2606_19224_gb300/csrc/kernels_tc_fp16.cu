// Instantiations of the mixed-precision persistent solve for FP16 operands (split from
// the BF16 ones so the two compile in parallel).
#include "tc_mixed.cuh"

namespace enkf {

template <bool PC, int TERMS>
static void* pick(int NT) {
  if (NT == 32) return (void*)solve_mixed_kernel<__half, 32, PC, TERMS>;
  if (NT == 64) return (void*)solve_mixed_kernel<__half, 64, PC, TERMS>;
  return (void*)solve_mixed_kernel<__half, 128, PC, TERMS>;
}

void* mixed_kernel_fp16(bool pc, bool split, int NT) {
  if (split) return pc ? pick<true, 3>(NT) : pick<false, 3>(NT);
  return pc ? pick<true, 1>(NT) : pick<false, 1>(NT);
}

}  // namespace enkf
