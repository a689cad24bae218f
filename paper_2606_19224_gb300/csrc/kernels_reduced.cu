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
//   reduced_cg_kernel      one CTA per column of M; G staged in shared memory; FP64 CG
//   update (kernels_fp.cu) X_a = X_f V (plain product mode)
//
// The same pass serves the paper's sEnKF comparator (Algorithm 3, the diagonal-inverse
// approximation): with the weights 1/s_i, s_i = |HA_i|^2 + (N-1) r_i (the diagonal of
// HA HA^T + R_N) instead of 1/r_i, and the innovation row D_i = Y~_i - HA_i as the only right
// factor (an N x N product per row instead of N x 2N), it forms
// W = sum_i HA_i^T D_i / s_i = HA^T diag(HA HA^T + R_N)^{-1} D, and X_a = X_f + A W (the
// CGD-EnKF update) with no solve at all.
#include "common.cuh"
#include "innov_device.cuh"
#include "gram_stages.cuh"

#include <algorithm>
#include <type_traits>

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

// A running product sum of the Gram pass: FP64 FMAs, or for double-float operands the
// compensated pair of DFAcc (exact FP32 products, TwoSum, errors gathered in c), renormalised
// every few terms. FP32 products of FP32-rounded anomalies would lose ~sqrt(m) in G's
// cancelling off-diagonals; double-float keeps about 44 bits at 12 FP32 operations per term,
// and FP32 issues at 64x the FP64 rate on this part.
template <typename AT> struct GramAcc;
template <> struct GramAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void renorm() {}
  __device__ __forceinline__ double value() const { return v; }
  __device__ __forceinline__ void set(double x) { v = x; }
};
template <> struct GramAcc<df32> {
  DFAcc d;
  __device__ __forceinline__ void add(const df32& a, const df32& b) { d.add(a, b); }
  __device__ __forceinline__ void renorm() { d.renorm(); }
  __device__ __forceinline__ double value() const { return (double)d.value(); }
  __device__ __forceinline__ void set(double x) {
    const df32 v(x);
    d.s = v.hi;
    d.c = v.lo;
  }
};

// VT: type of X_f; AT: type of the staged tiles and the accumulators: FP64 for FP64
// ensembles, double-float for FP32 ensembles (see GramAcc).
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
  constexpr int QN = NT / 32;                 // members per lane in the gather (j = lane + 32 q)
  constexpr int QP = (NT + 63) / 64;          // perturbation pairs per lane (p = lane + 32 qp)
  __shared__ __align__(16) AT sK[TR][NT];            // HA_i / r_i (sEnKF: HA_i / s_i)
  __shared__ __align__(16) AT sJ[TR][JW];            // [HA_i | Y~_i] (sEnKF: D_i)
  __shared__ double sred[RG > 1 ? TILES * 16 : 1];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int g = t / (kThreads / RG);                 // row group of this thread
  const int kbase = blockIdx.y * KR;
  GramAcc<AT> acc[TPT][4][4];   // zero-initialised

  const double inv_n = 1.0 / (double)N;   // FP64 divisions run on the same pipe as the Gram's
                                           // FMAs: one per thread here, one per row below
  const int64_t rows_per = (m + gridDim.x - 1) / gridDim.x;
  const int64_t row0 = min(m, (int64_t)blockIdx.x * rows_per);
  const int64_t row1 = min(m, row0 + rows_per);
  for (int64_t i0 = row0; i0 < row1; i0 += TR) {
    __syncthreads();
    // gather + anomalies + perturbed innovation-mean form: one warp per row of the tile
    for (int ii = warp; ii < TR; ii += kThreads / 32) {
      const int64_t i = i0 + ii;
      double z[QN];
#pragma unroll
      for (int q = 0; q < QN; ++q) z[q] = 0.0;
      if (i < row1) {
        const int k0 = rowptr[i], k1 = rowptr[i + 1];
        for (int k = k0; k < k1; ++k) {
          const double wk = w[k];
          const VT* xr = Xf + (int64_t)col[k] * N;
#pragma unroll
          for (int q = 0; q < QN; ++q) {
            const int j = lane + 32 * q;
            if (j < N) z[q] = fma(wk, (double)xr[j], z[q]);
          }
        }
      }
      double s = z[0];
#pragma unroll
      for (int q = 1; q < QN; ++q) s += z[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      const double zbar = s * inv_n;
      const double ri = i < row1 ? r[i] : 1.0;
      const double yi = i < row1 ? y[i] : 0.0;
      const double sr = (emode == 2) ? sqrt(ri) : 0.0;
      // perturbation pair p (members 2p, 2p + 1) is drawn once, by lane p % 32 in slot p / 32
      // (FP64 Box-Muller for FP64 ensembles, FP32 for FP32 ensembles, as in the innovations),
      // and handed to its two members' lanes with shuffles below
      double pr[QP][2];
#pragma unroll
      for (int qp = 0; qp < QP; ++qp) pr[qp][0] = pr[qp][1] = 0.0;
      if (emode == 2 && i < row1) {
#pragma unroll
        for (int qp = 0; qp < QP; ++qp) {
          const int jp = 2 * (lane + 32 * qp);
          if (jp < N) {
            if constexpr (sizeof(VT) == 4) perturbation_pair_f32(i, jp, seed, counter, pr[qp][0], pr[qp][1]);
            else perturbation_pair(i, jp, seed, counter, pr[qp][0], pr[qp][1]);
          }
        }
      }
      double ha[QN], yt[QN];
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const int j = lane + 32 * q;
        // member j belongs to pair 16 q + (lane >> 1): lane 16 (q & 1) + (lane >> 1), slot q >> 1
        const int src = 16 * (q & 1) + (lane >> 1);
        const double n_even = __shfl_sync(0xffffffffu, pr[q >> 1][0], src);
        const double n_odd = __shfl_sync(0xffffffffu, pr[q >> 1][1], src);
        ha[q] = 0.0;
        yt[q] = 0.0;
        if (i < row1 && j < N) {
          double pert = 0.0;
          if (emode == 1) pert = E[i * N + j];
          else if (emode == 2) pert = sr * ((lane & 1) ? n_odd : n_even);
          ha[q] = z[q] - zbar;
          yt[q] = (yi - zbar) + pert;
        }
      }
      double wgt = ri;   // the row's weight divisor: r_i, or s_i = |HA_i|^2 + (N-1) r_i
      if (SENKF) {
        double hn = ha[0] * ha[0];
#pragma unroll
        for (int q = 1; q < QN; ++q) hn = fma(ha[q], ha[q], hn);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) hn += __shfl_xor_sync(0xffffffffu, hn, o);
        wgt = hn + (double)(N - 1) * ri;
      }
      const double inv_w = 1.0 / wgt;
#pragma unroll
      for (int q = 0; q < QN; ++q) {
        const int j = lane + 32 * q;   // < NT
        sK[ii][j] = (AT)(ha[q] * inv_w);
        if (SENKF) {
          sJ[ii][j] = (AT)(yt[q] - ha[q]);
        } else {
          sJ[ii][j] = (AT)ha[q];
          sJ[ii][NT + j] = (AT)yt[q];
        }
      }
    }
    __syncthreads();
    const int nrows = (int)min((int64_t)TR, row1 - i0);
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
      const int u = (RG > 1) ? t % TILES : t + q * kThreads;
      const int tj = u % JG, tk = u / JG;
      int terms = 0;
      for (int ii = g; ii < nrows; ii += RG) {
        AT a[4], b[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = sK[ii][kbase + tk * 4 + x];
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) b[yy] = sJ[ii][tj * 4 + yy];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) acc[q][x][yy].add(a[x], b[yy]);
        if ((++terms & 3) == 0) {
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int yy = 0; yy < 4; ++yy) acc[q][x][yy].renorm();
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int yy = 0; yy < 4; ++yy) acc[q][x][yy].renorm();
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
          for (int yy = 0; yy < 4; ++yy) sred[u * 16 + x * 4 + yy] = acc[0][x][yy].value();
      }
      __syncthreads();
      if (g == 0) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int yy = 0; yy < 4; ++yy) acc[0][x][yy].set(acc[0][x][yy].value() + sred[t * 16 + x * 4 + yy]);
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
        if (k < N && j < N) out[(int64_t)half * N * N + k * N + j] = acc[q][x][yy].value();
      }
  }
}

// Fixed-order sum over b < nparts of part[b * pstride + e], e < count: a CTA takes 32
// consecutive e (one per lane), warp w adds b = w, w + 8, ... in order, and warp 0 adds the
// eight warp sums in warp order before handing (e, total) to store.
template <typename Store>
__device__ __forceinline__ void sum_partials(const double* __restrict__ part, int nparts,
                                             int64_t pstride, int count, Store&& store) {
  constexpr int W = kThreads / 32;
  __shared__ double wsum[W][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (e < count)
    for (int b = warp; b < nparts; b += W) s += part[(int64_t)b * pstride + e];
  wsum[warp][lane] = s;
  __syncthreads();
  if (warp == 0 && e < count) {
    double tot = wsum[0][lane];
#pragma unroll
    for (int q = 1; q < W; ++q) tot += wsum[q][lane];
    store(e, tot);
  }
}

// G = I + sum_b part_b[0] / (N-1), M = I + sum_b part_b[1] / (N-1).
__global__ void __launch_bounds__(kThreads) reduced_sum_kernel(const double* __restrict__ part, int nparts, int N,
                                                               double* __restrict__ Gm, double* __restrict__ Mm) {
  const int NN = N * N;
  const double inv = 1.0 / (double)(N - 1);
  sum_partials(part, nparts, 2 * (int64_t)NN, 2 * NN, [&](int e, double s) {
    const int half = e / NN, ee = e % NN;
    (half == 0 ? Gm : Mm)[ee] = s * inv + ((ee / N) == (ee % N) ? 1.0 : 0.0);
  });
}

// sEnKF: W = sum_b part_b[0] (= HA^T diag^{-1} D).
__global__ void __launch_bounds__(kThreads) senkf_sum_kernel(const double* __restrict__ part, int nparts, int N,
                                                             double* __restrict__ W) {
  sum_partials(part, nparts, 2 * (int64_t)N * N, N * N, [&](int e, double s) { W[e] = s; });
}

// One CTA per column j of M: CG for G v_j = m_j (FP64), G staged in shared memory.
// V is [N][N] row-major (V[k][j]).
__global__ void __launch_bounds__(kThreads) reduced_cg_kernel(
    const double* __restrict__ Gm, const double* __restrict__ Mm, int N, double tol, int max_iter,
    int fixed_iters, double* __restrict__ V, int* __restrict__ col_iters,
    double* __restrict__ col_relres, double* __restrict__ col_true, int* __restrict__ status) {
  extern __shared__ __align__(16) double sm[];
  // G with row stride N + 1: lanes on consecutive rows k then read distinct banks
  const int ld = N + 1;
  double* sG = sm;                 // N x (N + 1)
  double* sx = sG + N * ld;        // N
  double* sr = sx + N;             // N
  double* sp = sr + N;             // N
  double* sq = sp + N;             // N
  double* sb = sq + N;             // N (right-hand side)
  double* spart = sb + N;          // [kThreads] partial row sums of the matvec
  __shared__ double red[kThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int j = blockIdx.x;
  for (int e = t; e < N * N; e += kThreads) sG[(e / N) * ld + e % N] = Gm[e];
  for (int k = t; k < N; k += kThreads) {
    const double b = Mm[k * N + j];
    sb[k] = b;
    sx[k] = 0.0;
    sr[k] = b;
    sp[k] = b;
  }
  __syncthreads();
  // block-wide sum, the same fixed-order tree in every warp (FP64 instructions are scarce on
  // this part, so the eight warp sums are folded by three shuffle steps, not a serial loop)
  auto block_sum = [&](double v) -> double {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = lane < kThreads / 32 ? red[lane] : 0.0;
#pragma unroll
    for (int o = kThreads / 64; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return __shfl_sync(0xffffffffu, s, 0);
  };
  // G u: thread t forms the partial sum of row k = t % NP over columns l = g, g + P, ...
  // (g = t / NP, P = kThreads / NP groups); row k's owner (thread k) adds the P partials in
  // a fixed order. Ends with the partials written and synchronised.
  const int NP = N <= 64 ? 64 : 128, P = kThreads / NP;
  auto matvec_partials = [&](const double* u) {
    const int k = t % NP, g = t / NP;
    double acc = 0.0;
    if (k < N)
      for (int l = g; l < N; l += P) acc = fma(sG[k * ld + l], u[l], acc);
    spart[t] = acc;
    __syncthreads();
  };
  auto row_of = [&](int k) -> double {
    double s = spart[k];
    for (int g = 1; g < P; ++g) s += spart[g * NP + k];
    return s;
  };
  double v = 0.0;
  for (int k = t; k < N; k += kThreads) v = fma(sb[k], sb[k], v);
  const double bn2 = block_sum(v);
  // |r| <= tol |b| compared in squares, with tol shrunk by 4 ulps so that a stop always gives
  // sqrt(rr / bn2) <= tol for the residual reported below
  const double tol_s = tol * (1.0 - 4.0 * 2.220446049250313e-16);
  const double stop2 = tol_s * tol_s * bn2;
  double rr = bn2;
  const bool fixed = fixed_iters > 0;
  const int limit = fixed ? fixed_iters : max_iter;
  int it = 0;
  bool active = rr > 0.0;
  for (; it < limit && active; ++it) {
    // q = G p
    matvec_partials(sp);
    v = 0.0;
    for (int k = t; k < N; k += kThreads) {
      const double qk = row_of(k);
      sq[k] = qk;
      v = fma(sp[k], qk, v);
    }
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
    else active = rr > stop2;
  }
  // true residual m_j - G v_j (FP64)
  __syncthreads();
  matvec_partials(sx);
  v = 0.0;
  for (int k = t; k < N; k += kThreads) {
    const double d = sb[k] - row_of(k);
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
  using AT = typename std::conditional<sizeof(VT) == 8, double, df32>::type;
  if (NT == 32)
    reduced_gram_kernel<VT, AT, 32, SENKF><<<dim3(grid, 32 / GramCfg<32>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  else if (NT == 64)
    reduced_gram_kernel<VT, AT, 64, SENKF><<<dim3(grid, 64 / GramCfg<64>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  else
    reduced_gram_kernel<VT, AT, 128, SENKF><<<dim3(grid, 128 / GramCfg<128>::KR), kThreads, 0, h->stream>>>(X, ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter, c.m, c.N, ws.Tpart);
  return cudaGetLastError();
}

int reduced_grid(const enkf_handle_s* h) {
  const int64_t tiles = (h->cfg.m + 31) / 32;
  return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)h->sms * 2));
}

cudaError_t launch_gram_stage(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                              int emode, uint64_t seed, uint64_t counter) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const bool senkf = c.variant == ENKF_SENKF;
  const int grid = reduced_grid(h);
  cudaError_t e = cudaMemsetAsync(ws.status, 0, 4 * sizeof(int32_t), h->stream);
  if (senkf) {   // no solve: the per-column statistics read back as 0 iterations, residual 0
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_iters, 0, sizeof(int32_t) * c.N, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_relres, 0, sizeof(double) * c.N, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.col_true, 0, sizeof(double) * c.N, h->stream);
  }
  if (e != cudaSuccess) return e;
  const bool f64 = c.precision == ENKF_FP64;
  if (senkf)
    return f64 ? gram_launch<double, true>(h, Xf, y, E, emode, seed, counter, grid)
               : gram_launch<float, true>(h, Xf, y, E, emode, seed, counter, grid);
  return f64 ? gram_launch<double, false>(h, Xf, y, E, emode, seed, counter, grid)
             : gram_launch<float, false>(h, Xf, y, E, emode, seed, counter, grid);
}

cudaError_t launch_nxn_stage(enkf_handle_s* h) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int grid = reduced_grid(h);
  if (c.variant == ENKF_SENKF) {
    const int NN = c.N * c.N;
    senkf_sum_kernel<<<(NN + 31) / 32, kThreads, 0, h->stream>>>(ws.Tpart, grid, c.N, ws.W);
    return cudaGetLastError();
  }
  double* Gm = ws.Tred;            // N x N
  double* Mm = ws.Wacc;            // N x N
  const int NN2 = 2 * c.N * c.N;
  reduced_sum_kernel<<<(NN2 + 31) / 32, kThreads, 0, h->stream>>>(ws.Tpart, grid, c.N, Gm, Mm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(double) * ((size_t)c.N * (c.N + 1) + 5 * c.N + kThreads);
  e = cudaFuncSetAttribute(reduced_cg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  reduced_cg_kernel<<<c.N, kThreads, smem, h->stream>>>(Gm, Mm, c.N, c.tol, c.max_iter, c.fixed_iters,
                                                       ws.W, ws.col_iters, ws.col_relres, ws.col_true,
                                                       ws.status);
  return cudaGetLastError();
}

cudaError_t launch_reduced(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                           int emode, uint64_t seed, uint64_t counter) {
  cudaError_t e = launch_gram_stage(h, Xf, y, E, emode, seed, counter);
  return e != cudaSuccess ? e : launch_nxn_stage(h);
}

}  // namespace enkf
