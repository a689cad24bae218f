// Tridiagonal observation-error covariance R (the noise model of the paper's Example 2:
// R_ii = sigma^2, R_{i,i+1} = R_{i+1,i} = sigma^2 rho; Sec. 5.3 and Sec. 6.2).
//
// With R = L L^T (L lower bidiagonal; its entries come from the banded Cholesky recurrence
// on the host, O(m) as Sec. 5.3 notes), the library analyses the whitened problem:
//
//   X' = L^{-1} HA   (m x N, zero-mean rows),  H' = I,  r' = 1,
//   y' = L^{-1} (y - zbar),                    E' = L^{-1} E  (or drawn as N(0, I)),
//
// which is exact for the two forms that use R only through L:
//   * CGD-EnKF-Reduced (Algorithm 2): P = L_N^{-1} HA with R_N = (N-1) R = L_N L_N^T, i.e.
//     P = X'/sqrt(N-1), and L_N^{-1}((y - zbar) 1^T + E) = (y' 1^T + E')/sqrt(N-1);
//   * CGD-EnKF with CG preconditioned by R: CG on L^{-1} S L^{-T} = X' X'^T/(N-1) + I for
//     Z' = L^T Z, with W = HA^T Z/(N-1) = X'^T Z'/(N-1) unchanged.
// The update X_a = X_f + A W (or X_f V) then uses the caller's X_f. Perturbations drawn
// inside the analysis are E' = xi (r' = 1), i.e. E = L xi ~ N(0, R).
//
// L^{-1} is a first-order linear recurrence over the rows, t_i = a_i u_i + b_i t_{i-1}
// (a_i = 1/L_ii, b_i = -L_{i,i-1}/L_ii), independent per column. It runs as a blocked scan:
// each block of kWhitenBlock rows solves its recurrence from a zero carry (whiten_scan),
// the carries into the blocks follow sequentially over the blocks (whiten_carry), and every
// row adds c_i times its block's carry-in, c_i the product of b over the block up to row i
// (whiten_fix): the same result as the sequential recurrence, in exact arithmetic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace enkf {

constexpr int kWhitenBlock = 256;   // rows per block of the scan

// Observed anomalies and the innovation mean, one warp per observation row:
// HA_i = (H X_f)_i - zbar_i into U[i][0..N), y_i - zbar_i into U[i][N] (FP64, row stride
// N + 1); with explicit perturbations, E_i into V[i][0..N).
template <typename VT>
__global__ void __launch_bounds__(kThreads) whiten_rows_kernel(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, int64_t m, int N,
    double* __restrict__ U) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const int S = N + 1;
  for (int64_t i = warp; i < m; i += nwarps) {
    const int k0 = rowptr[i], k1 = rowptr[i + 1];
    double z[4] = {0.0, 0.0, 0.0, 0.0};   // members lane, lane + 32, lane + 64, lane + 96
    for (int k = k0; k < k1; ++k) {
      const double wk = w[k];
      const VT* xr = Xf + (int64_t)col[k] * N;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        if (j < N) z[q] = fma(wk, (double)xr[j], z[q]);
      }
    }
    double s = z[0] + z[1] + z[2] + z[3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double zbar = s / (double)N;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = lane + 32 * q;
      if (j < N) U[i * S + j] = z[q] - zbar;
    }
    if (lane == 0) U[i * S + N] = y[i] - zbar;
  }
}

// Local recurrence of every block from a zero carry, in place, for C columns of a row-major
// [m][C] array; the block's last value into carry[blk][c]. One thread per column, one CTA
// per block.
__global__ void whiten_scan_kernel(double* __restrict__ U, int64_t m, int C, const double* __restrict__ a,
                                   const double* __restrict__ b, double* __restrict__ carry) {
  const int c = threadIdx.x;
  const int64_t blk = blockIdx.x;
  const int64_t i0 = blk * kWhitenBlock;
  const int64_t i1 = i0 + kWhitenBlock < m ? i0 + kWhitenBlock : m;
  if (c >= C) return;
  double t = 0.0;
#pragma unroll 8
  for (int64_t i = i0; i < i1; ++i) {
    t = fma(b[i], t, a[i] * U[i * C + c]);
    U[i * C + c] = t;
  }
  carry[blk * C + c] = t;
}

// Carries into the blocks: carry_in[0] = 0, carry_in[k+1] = end[k] + mu[k] carry_in[k], with
// end[k] the block's local last value (overwritten in place by the carry-in).
__global__ void whiten_carry_kernel(double* __restrict__ carry, int64_t nblk, int C,
                                    const double* __restrict__ mu) {
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    double prev = 0.0;
    for (int64_t k = 0; k < nblk; ++k) {
      const double end = carry[k * C + c];
      carry[k * C + c] = prev;
      prev = fma(mu[k], prev, end);
    }
  }
}

// Row i of block k: t_i += cp_i carry_in[k]. Columns [0, N) go to the whitened ensemble Xw
// (in VT), column N of U to y' (FP64), and, when E is given, the N columns of V to E' (Ew
// may be V itself: each entry is read and written by the same thread).
template <typename VT>
__global__ void __launch_bounds__(kThreads) whiten_fix_kernel(
    const double* __restrict__ U, const double* __restrict__ carryU, const double* __restrict__ V,
    const double* __restrict__ carryV, const double* __restrict__ cp, int64_t m, int N, VT* __restrict__ Xw,
    double* __restrict__ yw, double* __restrict__ Ew) {
  const int S = N + 1;
  const int64_t total = m * S;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total; e += (int64_t)gridDim.x * kThreads) {
    const int64_t i = e / S;
    const int c = (int)(e % S);
    const int64_t k = i / kWhitenBlock;
    const double v = fma(cp[i], carryU[k * S + c], U[e]);
    if (c < N) Xw[i * N + c] = (VT)v;
    else yw[i] = v;
    if (V != nullptr && c < N) Ew[i * N + c] = fma(cp[i], carryV[k * N + c], V[i * N + c]);
  }
}

// ------------------------------------------------------------------ host side
// Banded Cholesky of the tridiagonal R (diagonal r, off-diagonal r_off) on the host and the
// scan coefficients; false if R is not positive definite.
bool whiten_coefficients(int64_t m, const double* r, const double* r_off, std::vector<double>& a,
                         std::vector<double>& b, std::vector<double>& cp, std::vector<double>& mu) {
  a.assign(m, 0.0);
  b.assign(m, 0.0);
  cp.assign(m, 0.0);
  const int64_t nblk = (m + kWhitenBlock - 1) / kWhitenBlock;
  mu.assign(nblk, 0.0);
  double lprev = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    double lo = 0.0, d = r[i];
    if (i > 0) {
      lo = r_off[i - 1] / lprev;
      d -= lo * lo;
    }
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double l = std::sqrt(d);
    a[i] = 1.0 / l;
    b[i] = -lo / l;
    // product of b over the block up to row i (the first row of a block starts a new product)
    cp[i] = (i % kWhitenBlock == 0) ? b[i] : cp[i - 1] * b[i];
    if (i % kWhitenBlock == kWhitenBlock - 1 || i == m - 1) mu[i / kWhitenBlock] = cp[i];
    lprev = l;
  }
  return true;
}

int64_t whiten_blocks(int64_t m) { return (m + kWhitenBlock - 1) / kWhitenBlock; }

cudaError_t launch_whiten(enkf_handle_s* h, const void* Xf, const double* y, const double* E) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int64_t m = c.m;
  const int N = c.N;
  const int S = N + 1;
  const int64_t nblk = whiten_blocks(m);
  const int rows_blocks = (int)std::min<int64_t>((m + 7) / 8, (int64_t)h->sms * 16);
  const bool f64 = c.precision == ENKF_FP64;
  if (f64)
    whiten_rows_kernel<double><<<rows_blocks, kThreads, 0, h->stream>>>(
        static_cast<const double*>(Xf), ws.Hrowptr, ws.Hcol, ws.Hw, y, m, N, ws.wU);
  else
    whiten_rows_kernel<float><<<rows_blocks, kThreads, 0, h->stream>>>(
        static_cast<const float*>(Xf), ws.Hrowptr, ws.Hcol, ws.Hw, y, m, N, ws.wU);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  whiten_scan_kernel<<<(unsigned)nblk, ((S + 31) / 32) * 32, 0, h->stream>>>(ws.wU, m, S, ws.wa, ws.wb, ws.wcarry);
  if (E) {
    e = cudaMemcpyAsync(ws.wV, E, sizeof(double) * m * N, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
    whiten_scan_kernel<<<(unsigned)nblk, ((N + 31) / 32) * 32, 0, h->stream>>>(ws.wV, m, N, ws.wa, ws.wb,
                                                                              ws.wcarryV);
  }
  whiten_carry_kernel<<<1, ((S + 31) / 32) * 32, 0, h->stream>>>(ws.wcarry, nblk, S, ws.wmu);
  if (E) whiten_carry_kernel<<<1, ((N + 31) / 32) * 32, 0, h->stream>>>(ws.wcarryV, nblk, N, ws.wmu);
  const int fix_blocks = (int)std::min<int64_t>((m * S + kThreads - 1) / kThreads, (int64_t)h->sms * 32);
  if (f64)
    whiten_fix_kernel<double><<<fix_blocks, kThreads, 0, h->stream>>>(
        ws.wU, ws.wcarry, E ? ws.wV : nullptr, ws.wcarryV, ws.wcp, m, N, static_cast<double*>(ws.Xw), ws.yw,
        ws.wV);
  else
    whiten_fix_kernel<float><<<fix_blocks, kThreads, 0, h->stream>>>(
        ws.wU, ws.wcarry, E ? ws.wV : nullptr, ws.wcarryV, ws.wcp, m, N, static_cast<float*>(ws.Xw), ws.yw,
        ws.wV);
  return cudaGetLastError();
}

}  // namespace enkf
