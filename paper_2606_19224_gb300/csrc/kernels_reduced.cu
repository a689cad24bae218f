// CGD-EnKF-Reduced (Sec. 5.2): Algorithm 2 with (I + P^T P)^{-1} applied by CG.
//
//   P = L^{-1} HA with L L^T = R_N = (N-1) R (L diagonal here), so
//   G = I + P^T P          = I + HA^T R^{-1} HA / (N-1)                  (N x N)
//   M = I + P^T L^{-1} Y~  = I + HA^T R^{-1} Y~ / (N-1),  Y~ = (y - zbar) 1^T + E
//   V = G^{-1} M by N independent CG recurrences (one per column of M), X_a = X_f V.
//
//   reduced_gram_kernel    one pass over the observation rows: gathers the rows of X_f that
//                          H touches, forms zbar, HA and Y~ for a tile of rows in shared
//                          memory, and accumulates this CTA's partial HA^T R^{-1} [HA | Y~]
//                          (the paper's "dominant cost ... formation of an N x N matrix",
//                          Sec. 6.2.2); HA and D are never written to HBM
//   reduced_sum_kernel     fixed-order sum of the CTA partials -> G, M (FP64)
//   reduced_cg_kernel      one CTA per group of columns; G staged in shared memory; FP64 CG
//   update (kernels_fp.cu) X_a = X_f V (plain product mode)
//
// The same pass serves the paper's sEnKF comparator (Algorithm 3, the diagonal-inverse
// approximation): with the weights 1/s_i, s_i = |HA_i|^2 + (N-1) r_i (the diagonal of
// HA HA^T + R_N) instead of 1/r_i, and the innovation row D_i = Y~_i - HA_i as the only right
// factor (an N x N product per row instead of N x 2N), it forms
// W = sum_i HA_i^T D_i / s_i = HA^T diag(HA HA^T + R_N)^{-1} D, and X_a = X_f + A W (the
// CGD-EnKF update) with no solve at all.
#include "common.cuh"
#include "senkf.cuh"

#include <algorithm>

namespace enkf {

// observation rows staged per tile: keeps the static tiles (3 NT values per row) <= 40 KB
template <typename VT, int NT> __host__ __device__ constexpr int red_tr() {
  constexpr int t = 40960 / (3 * NT * (int)sizeof(VT));
  return t >= 32 ? 32 : (t / 8) * 8;
}

// Gram pass. CTA (bx, ks) accumulates, over its block of observation rows, the rows
// k in [ks*KR, (ks+1)*KR) of HA^T R^{-1} [HA | Y~] (an N x 2N product; sEnKF:
// HA^T diag^{-1} D, N x N) with a 4x4 register tile per thread; gridDim.y = NT/KR splits k so
// that a thread keeps at most 32 accumulators.
template <int NT> struct GramCfg;
template <> struct GramCfg<32> { static constexpr int KR = 32; };
template <> struct GramCfg<64> { static constexpr int KR = 64; };
template <> struct GramCfg<128> { static constexpr int KR = 32; };

// VT: type of X_f; AT: type of the staged tiles and the accumulators (FP64 in both modes:
// FP32 products of FP32-rounded anomalies lose ~sqrt(m) in the cancelling off-diagonals).
template <typename VT, typename AT, int NT, bool SENKF = false>
__global__ void __launch_bounds__(kThreads) reduced_gram_kernel(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ part /* [gridDim.x][2][N][N]; sEnKF writes only [b][0] */) {
  constexpr int KR = GramCfg<NT>::KR;
  constexpr int JW = SENKF ? NT : 2 * NT;                          // columns of the right factor
  constexpr int KG = KR / 4, JG = JW / 4, TILES = KG * JG;
  constexpr int TPT = TILES >= kThreads ? TILES / kThreads : 1;   // tiles per thread
  constexpr int RG = TILES >= kThreads ? 1 : kThreads / TILES;    // row groups
  static_assert(TILES % kThreads == 0 || kThreads % TILES == 0, "mapping");
  constexpr int TR = red_tr<AT, NT>();
  __shared__ __align__(16) AT sK[TR][NT];            // HA_i / r_i (sEnKF: HA_i / s_i)
  __shared__ __align__(16) AT sJ[TR][JW];            // [HA_i | Y~_i] (sEnKF: D_i)
  __shared__ double sred[RG > 1 ? TILES * 16 : 1];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = t / (kThreads / RG);                 // row group of this thread
  const int kbase = blockIdx.y * KR;
  AT acc[TPT][4][4];
#pragma unroll
  for (int q = 0; q < TPT; ++q)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) acc[q][x][yy] = AT(0);

  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t row0 = min(m, (int64_t)blockIdx.x * rows_per);
  const int64_t row1 = min(m, row0 + rows_per);
  for (int64_t i0 = row0; i0 < row1; i0 += TR) {
    __syncthreads();
    // gather + anomalies + perturbed innovation-mean form: one warp per row of the tile
    for (int ii = warp; ii < TR; ii += kThreads / 32) {
      const int64_t i = i0 + ii;
      double z[4] = {0.0, 0.0, 0.0, 0.0};
      if (i < row1) {
        const int k0 = rowptr[i], k1 = rowptr[i + 1];
        for (int k = k0; k < k1; ++k) {
          const double wk = w[k];
          const VT* xr = Xf + (int64_t)col[k] * N;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = lane + 32 * q;
            if (j < N) z[q] = fma(wk, (double)xr[j], z[q]);
          }
        }
      }
      double s = z[0] + z[1] + z[2] + z[3];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double zbar = s / (double)N;
      const double ri = i < row1 ? r[i] : 1.0;
      const double yi = i < row1 ? y[i] : 0.0;
      const double sr = sqrt(ri);
      double ha[4], yt[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        ha[q] = 0.0;
        yt[q] = 0.0;
        if (i < row1 && j < N) {
          double pert = 0.0;
          if (emode == 1) pert = E[i * N + j];
          else if (emode == 2) pert = sr * perturbation_normal(i, j, seed, counter);
          ha[q] = z[q] - zbar;
          yt[q] = (yi - zbar) + pert;
        }
      }
      double wgt = ri;   // the row's weight divisor: r_i, or s_i = |HA_i|^2 + (N-1) r_i
      if (SENKF) {
        double hn = ha[0] * ha[0] + ha[1] * ha[1] + ha[2] * ha[2] + ha[3] * ha[3];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hn += __shfl_xor_sync(0xffffffffu, hn, o);
        wgt = hn + (double)(N - 1) * ri;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = lane + 32 * q;
        if (j < NT) {
          sK[ii][j] = (AT)(ha[q] / wgt);
          if (SENKF) {
            sJ[ii][j] = (AT)(yt[q] - ha[q]);
          } else {
            sJ[ii][j] = (AT)ha[q];
            sJ[ii][NT + j] = (AT)yt[q];
          }
        }
      }
    }
    __syncthreads();
    const int nrows = (int)min((int64_t)TR, row1 - i0);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int u = (RG > 1) ? t % TILES : t + q * kThreads;
      const int tj = u % JG, tk = u / JG;
      for (int ii = g; ii < nrows; ii += RG) {
        AT a[4], b[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = sK[ii][kbase + tk * 4 + x];
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) b[yy] = sJ[ii][tj * 4 + yy];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) acc[q][x][yy] = fma(a[x], b[yy], acc[q][x][yy]);
      }
    }
  }
  // fold the row groups (fixed order) and write this CTA's partial rows (FP64)
  if (RG > 1) {
    __syncthreads();
    for (int gg = 1; gg < RG; ++gg) {
      if (g == gg) {
        const int u = t % TILES;
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) sred[u * 16 + x * 4 + yy] = (double)acc[0][x][yy];
      }
      __syncthreads();
      if (g == 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) acc[0][x][yy] = (AT)((double)acc[0][x][yy] + sred[t * 16 + x * 4 + yy]);
      }
      __syncthreads();
    }
  }
  if (RG > 1 && g != 0) return;
  double* out = part + (int64_t)blockIdx.x * 2 * N * N;
#pragma unroll
  for (int q = 0; q < TPT; ++q) {
    const int u = (RG > 1) ? t % TILES : t + q * kThreads;
    const int tj = u % JG, tk = u / JG;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int yy = 0; yy < 4; ++yy) {
        const int k = kbase + tk * 4 + x, jj = tj * 4 + yy;
        const int half = jj / NT, j = jj % NT;
        if (k < N && j < N) out[(int64_t)half * N * N + k * N + j] = (double)acc[q][x][yy];
      }
  }
}

// G = I + sum_b part_b[0] / (N-1), M = I + sum_b part_b[1] / (N-1), fixed order over b.
__global__ void reduced_sum_kernel(const double* __restrict__ part, int nparts, int N,
                                   double* __restrict__ Gm, double* __restrict__ Mm) {
  const int NN = N * N;
  const double inv = 1.0 / (double)(N - 1);
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < 2 * NN; e += gridDim.x * kThreads) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * 2 * NN + e];
    const int half = e / NN, ee = e % NN;
    const double v = s * inv + ((ee / N) == (ee % N) ? 1.0 : 0.0);
    (half == 0 ? Gm : Mm)[ee] = v;
  }
}

// sEnKF: W = sum_b part_b[0] (= HA^T diag^{-1} D), fixed order over b.
__global__ void senkf_sum_kernel(const double* __restrict__ part, int nparts, int N, double* __restrict__ W) {
  const int NN = N * N;
  for (int e = blockIdx.x * kThreads + threadIdx.x; e < NN; e += gridDim.x * kThreads) {
    double a = 0.0;
    for (int q = 0; q < nparts; ++q) a += part[(int64_t)q * 2 * NN + e];
    W[e] = a;
  }
}

// One CTA per column j of M: CG for G v_j = m_j (FP64), G staged in shared memory.
// V is [N][N] row-major (V[k][j]).
__global__ void __launch_bounds__(kThreads) reduced_cg_kernel(
    const double* __restrict__ Gm, const double* __restrict__ Mm, int N, double tol, int max_iter,
    int fixed_iters, double* __restrict__ V, int* __restrict__ col_iters,
    double* __restrict__ col_relres, double* __restrict__ col_true, int* __restrict__ status) {
  extern __shared__ __align__(16) double sm[];
  double* sG = sm;                 // N x N
  double* sx = sG + N * N;         // N
  double* sr = sx + N;             // N
  double* sp = sr + N;             // N
  double* sq = sp + N;             // N
  double* sb = sq + N;             // N (right-hand side)
  __shared__ double red[kThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int j = blockIdx.x;
  for (int e = t; e < N * N; e += kThreads) sG[e] = Gm[e];
  for (int k = t; k < N; k += kThreads) {
    const double b = Mm[k * N + j];
    sb[k] = b;
    sx[k] = 0.0;
    sr[k] = b;
    sp[k] = b;
  }
  __syncthreads();
  auto block_sum = [&](double v) -> double {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[q];
    return s;
  };
  double v = 0.0;
  for (int k = t; k < N; k += kThreads) v = fma(sb[k], sb[k], v);
  const double bn2 = block_sum(v);
  double rr = bn2;
  const bool fixed = fixed_iters > 0;
  const int limit = fixed ? fixed_iters : max_iter;
  int it = 0;
  bool active = rr > 0.0;
  for (; it < limit && active; ++it) {
    // q = G p
    for (int k = t; k < N; k += kThreads) {
      double s = 0.0;
      for (int l = 0; l < N; ++l) s = fma(sG[k * N + l], sp[l], s);
      sq[k] = s;
    }
    __syncthreads();
    v = 0.0;
    for (int k = t; k < N; k += kThreads) v = fma(sp[k], sq[k], v);
    const double pq = block_sum(v);
    if (!(pq > 0.0) || !isfinite(pq)) {
      if (t == 0) atomicOr(status, isfinite(pq) ? DS_BREAKDOWN : DS_NONFINITE);
      break;
    }
    const double alpha = rr / pq;
    v = 0.0;
    for (int k = t; k < N; k += kThreads) {
      sx[k] = fma(alpha, sp[k], sx[k]);
      const double rn = fma(-alpha, sq[k], sr[k]);
      sr[k] = rn;
      v = fma(rn, rn, v);
    }
    const double rn2 = block_sum(v);
    const double beta = rn2 / rr;
    rr = rn2;
    for (int k = t; k < N; k += kThreads) sp[k] = fma(beta, sp[k], sr[k]);
    __syncthreads();
    if (fixed) active = rr > 0.0;
    else active = sqrt(rr) > tol * sqrt(bn2);
  }
  // true residual m_j - G v_j (FP64)
  v = 0.0;
  for (int k = t; k < N; k += kThreads) {
    double s = 0.0;
    for (int l = 0; l < N; ++l) s = fma(sG[k * N + l], sx[l], s);
    const double d = sb[k] - s;
    v = fma(d, d, v);
  }
  const double tr2 = block_sum(v);
  for (int k = t; k < N; k += kThreads) V[k * N + j] = sx[k];
  if (t == 0) {
    col_iters[j] = it;
    const double rel = bn2 > 0.0 ? sqrt(rr / bn2) : 0.0;
    col_relres[j] = rel;
    col_true[j] = bn2 > 0.0 ? sqrt(tr2 / bn2) : 0.0;
    if (!fixed && !(rel <= tol)) atomicOr(status, DS_NOT_CONVERGED);
  }
}

// ------------------------------------------------------------------ launchers
template <typename VT, bool SENKF>
static cudaError_t gram_launch(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                               int emode, uint64_t seed, uint64_t counter, int grid) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int NT = c.N <= 32 ? 32 : (c.N <= 64 ? 64 : 128);
  const VT* X = static_cast<const VT*>(Xf);
  if (NT == 32)
    reduced_gram_kernel<VT, double, 32, SENKF><<<dim3(grid, 32 / GramCfg<32>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  else if (NT == 64)
    reduced_gram_kernel<VT, double, 64, SENKF><<<dim3(grid, 64 / GramCfg<64>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  else
    reduced_gram_kernel<VT, double, 128, SENKF><<<dim3(grid, 128 / GramCfg<128>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  return cudaGetLastError();
}

int reduced_grid(const enkf_handle_s* h) {
  const int64_t tiles = (h->cfg.m + 31) / 32;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)h->sms * 2));
}

cudaError_t launch_reduced(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                           int emode, uint64_t seed, uint64_t counter) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int grid = reduced_grid(h);
  cudaError_t e = cudaMemsetAsync(ws.status, 0, 4 * sizeof(int32_t), h->stream);
  if (e != cudaSuccess) return e;
  e = c.precision == ENKF_FP64 ? gram_launch<double, false>(h, Xf, y, E, emode, seed, counter, grid)
                               : gram_launch<float, false>(h, Xf, y, E, emode, seed, counter, grid);
  if (e != cudaSuccess) return e;
  double* Gm = ws.Tred;            // N x N
  double* Mm = ws.Wacc;            // N x N
  const int NN2 = 2 * c.N * c.N;
  reduced_sum_kernel<<<(NN2 + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(ws.Tpart, grid, c.N, Gm, Mm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(double) * ((size_t)c.N * c.N + 5 * c.N);
  e = cudaFuncSetAttribute(reduced_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  reduced_cg_kernel<<<c.N, kThreads, smem, h->stream>>>(Gm, Mm, c.N, c.tol, c.max_iter, c.fixed_iters,
                                                       ws.W, ws.col_iters, ws.col_relres, ws.col_true,
                                                       ws.status);
  return cudaGetLastError();
}

cudaError_t launch_senkf(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                         int emode, uint64_t seed, uint64_t counter) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int grid = reduced_grid(h);
  cudaError_t e = cudaMemsetAsync(ws.status, 0, 4 * sizeof(int32_t), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_iters, 0, sizeof(int32_t) * c.N, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_relres, 0, sizeof(double) * c.N, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_true, 0, sizeof(double) * c.N, h->stream);
  if (e != cudaSuccess) return e;
  e = c.precision == ENKF_FP64 ? gram_launch<double, true>(h, Xf, y, E, emode, seed, counter, grid)
                               : gram_launch<float, true>(h, Xf, y, E, emode, seed, counter, grid);
  if (e != cudaSuccess) return e;
  const int NN = c.N * c.N;
  senkf_sum_kernel<<<(NN + kThreads - 1) / kThreads, kThreads, 0, h->stream>>>(ws.Tpart, grid, c.N, ws.W);
  return cudaGetLastError();
}

}  // namespace enkf
