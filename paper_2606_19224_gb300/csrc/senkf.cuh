// The paper's sEnKF comparator (Algorithm 3), built from the Reduced variant's Gram pass
// (kernels_reduced.cu) and the CGD-EnKF update.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct enkf_handle_s;

namespace enkf {
// W = HA^T diag(HA HA^T + R_N)^{-1} D into ws.W (R_N = (N-1) R), no solve; the CTA partials
// use ws.Tpart ([reduced_grid][2 N N]). The caller then applies X_a = X_f + A W.
cudaError_t launch_senkf(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                         int emode, uint64_t seed, uint64_t counter);
}  // namespace enkf
