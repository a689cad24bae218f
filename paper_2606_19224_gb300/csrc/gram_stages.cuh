// The two stages of the variants built on one Gram pass over the observation rows
// (kernels_reduced.cu): CGD-EnKF-Reduced (Algorithm 2 with the N x N inverse applied by CG)
// and the paper's sEnKF comparator (Algorithm 3, the diagonal-inverse approximation). The
// analysis call times them as two phases, then applies the update.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct enkf_handle_s;

namespace enkf {
// Gram pass into ws.Tpart ([reduced_grid][2 N N] FP64 partials). Reduced: HA^T R^{-1} [HA | Y~]
// per CTA; sEnKF: HA^T diag(HA HA^T + R_N)^{-1} D per CTA (R_N = (N-1) R, slot 0 only).
cudaError_t launch_gram_stage(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                              int emode, uint64_t seed, uint64_t counter);
// N x N stage. Reduced: G, M from the partials, CG on G V = M (V into ws.W, G in ws.Tred).
// sEnKF: W = sum of the partials into ws.W (X_a = X_f + A W), no solve.
cudaError_t launch_nxn_stage(enkf_handle_s* h);
}  // namespace enkf
