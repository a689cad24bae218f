// CUDA kernels of the CGD-EnKF analysis step on CUDA cores (FP64 and FP32 paths).
//
//   innov_kernel   Z_obs = H X_f (CSR gather), zbar, HA = Z_obs - zbar 1^T, E (Philox or given),
//                  D = y 1^T - Z_obs + E                         (Sec. 2.3, Eq. Zhat_def)
//   solve_kernel   persistent cooperative CG on S Z = D with S V = HA (HA^T V)/(N-1) + R V
//                  (Sec. 3.3, Eq. matvec_decomp); N independent recurrences share each
//                  matvec; FP64 scalars; FP32 mode = FP32 inner solves + FP64 residual
//                  refresh (iterative refinement), all on the device in one launch
//   update_kernel  X_a = X_f + A W, W = HA^T Z/(N-1), A = X_f - xbar 1^T  (Fig. 2, Alg. 1)
//
// Data layout: every [rows][N] array is row-major with the member index fastest. The
// persistent grid splits the m observation rows into contiguous blocks, one per CTA (the
// paper's row-block distribution, Sec. 3.3, with CTAs in place of MPI ranks); the only
// cross-CTA traffic per CG step is the N x N partial Gram T = HA^T P (+ N values of
// sum r p^2) and N residual norms, reduced in a fixed order so results are bitwise
// reproducible run to run.
//
// Element work is done on 4-column fragments (one 128-bit access for FP32, two for FP64
// when N % 4 == 0), and the operands of each pass-B epilogue are loaded before the
// contraction so their latency overlaps it. In the FP32 mode the inner loops contain no
// FP64 arithmetic (FP64 runs at 1/64 of the FP32 rate on this part): per-thread partial
// sums are FP32 and only the cross-thread / cross-CTA reductions and the CG scalars are FP64.
#include "cg_device.cuh"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

namespace enkf {

struct SolveParams {
  int64_t m;
  int N;
  int mode;  // 0: FP64 CG (X is the FP64 solution Z); 1: FP32 inner CG + FP64 refresh
  const void* HA;
  const double* HA64;
  const double* D;
  const double* r;
  const void* rv;   // r in the inner-solve type
  void* B;
  void* X;
  void* Res;
  void* P;
  void* Sv;
  double* Z;
  const df32* HAdf;   // HA and D in double-float, and the double-float solution (FP32 mode)
  const df32* Ddf;
  df32* Zdf;
  double* Tpart;
  double* Tred;
  double* rrpart;
  double* W;
  double tol, inner_tol;
  int max_iter, fixed_iters, max_refine, true_residual;
  int* col_iters;
  double* col_relres;
  double* col_true;
  int* status;
  unsigned* bar;
  unsigned long long* prof;  // optional phase timers of CTA 0 (ns), nullptr when off
};

// Phase timer slots (CTA 0, thread 0): accumulated ns per phase of the solve.
enum : int { PH_SETUP = 0, PH_PASS, PH_BAR1, PH_RED, PH_BAR2, PH_SCAL, PH_REFRESH, PH_COUNT = 8 };

template <typename VT, int NT, bool PC>
__global__ void __launch_bounds__(kThreads, ((NT == 128 || (NT == 64 && sizeof(VT) == 8)) ? 1 : 2)) solve_kernel(SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* s_gam = reinterpret_cast<double*>(smem);   // (r, r) of the current residual
  double* s_gold = s_gam + NT;                        // previous (r, r)
  double* s_sig = s_gold + NT;                        // sum r_i r_ij^2
  double* s_tn2 = s_sig + NT;                         // ||HA^T r_j||^2
  double* s_bn2 = s_tn2 + NT;                         // ||b_j||^2 of the inner solve
  double* s_dn2 = s_bn2 + NT;                         // ||d_j||^2
  double* s_alpha = s_dn2 + NT;
  double* s_beta = s_alpha + NT;
  double* s_itol = s_beta + NT;
  double* s_tmp = s_itol + NT;
  double* s_true = s_tmp + NT;
  double* s_spare = s_true + NT;
  int* s_active = reinterpret_cast<int*>(s_spare + NT);
  int* s_done = s_active + NT;
  int* s_iters = s_done + NT;
  int* s_flag = s_iters + NT;
  VT* s_alpha_v = reinterpret_cast<VT*>(s_flag + NT);
  VT* s_beta_v = reinterpret_cast<VT*>(reinterpret_cast<unsigned char*>(s_flag + NT) + NT * 8);
  double* scratch = reinterpret_cast<double*>(smem + scalar_bytes<NT>());
  unsigned char* uni = smem + scalar_bytes<NT>() + kThreads * 8;
  constexpr int LDV = NT + 16 / (int)sizeof(VT);
  VT* sT = reinterpret_cast<VT*>(uni);
  unsigned char* tiles = uni + NT * LDV * sizeof(VT);

  const int N = p.N, G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int64_t rows_per = (p.m + G - 1) / G;
  const int64_t row0 = imin64(p.m, (int64_t)b * rows_per);
  const int64_t row1 = imin64(p.m, row0 + rows_per);
  const int NE = N * N + 2 * N;
  GridBarrier bar{p.bar, reinterpret_cast<int*>(p.bar + 1), p.status, (unsigned)G, 0u};
  const double inv_nm1 = 1.0 / (double)(N - 1);
  const bool refine = (p.mode == 1);
  const bool fixed = p.fixed_iters > 0;
  VT* X = refine ? static_cast<VT*>(p.X) : reinterpret_cast<VT*>(p.Z);
  VT* Res = static_cast<VT*>(p.Res);
  VT* P = static_cast<VT*>(p.P);
  VT* Sv = static_cast<VT*>(p.Sv);
  const VT* B = refine ? static_cast<const VT*>(p.B) : reinterpret_cast<const VT*>(p.D);
  const VT* HA = static_cast<const VT*>(p.HA);
  const VT* rv = static_cast<const VT*>(p.rv);
  double* Tp = p.Tpart + (int64_t)b * NE;
  const bool prof = p.prof != nullptr && b == 0 && t == 0;
  unsigned long long ph[PH_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long tp = prof ? global_ns() : 0ull;
  auto tick = [&](int slot) {
    if (prof) {
      const unsigned long long now = global_ns();
      ph[slot] += now - tp;
      tp = now;
    }
  };
  int par = 0;
  bool ok = true;

  // ---- ||d_j||^2 (and Z = 0 for the refinement accumulator)
  rows_reduce<NT>(row0, row1, N, [&](int64_t i, int j, double& acc) {
    const double d = p.D[i * N + j];
    acc = fma(d, d, acc);
    if (refine) p.Zdf[i * N + j] = df32(0.f, 0.f);
  }, s_tmp, scratch);
  if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
  ok = bar.sync();
  if (ok) {
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_dn2, scratch);
    par ^= 1;
    if (t < NT) {
      const bool zero = (t >= N) || (s_dn2[t] == 0.0);
      s_done[t] = zero ? 1 : 0;
      s_iters[t] = 0;
      s_true[t] = (t < N && s_dn2[t] == 0.0) ? 0.0 : -1.0;
      s_gam[t] = 0.0;
      s_bn2[t] = 0.0;
      s_itol[t] = refine ? p.inner_tol : p.tol;
      s_alpha_v[t] = VT(0);
      s_beta_v[t] = VT(0);
    }
    __syncthreads();
  }
  tick(PH_SETUP);

  int outer = 0, total_iter = 0, refinements = 0;
  while (ok) {
    // ---- inner solve of S X = B from X = 0: first reduction of [HA^T r | sum r_i r^2 | (r, r)]
    {
      ProSetup<VT, PC> pro{B, X, Res, rv, N};
      passA<VT, NT, ProSetup<VT, PC>, PC>(HA, row0, row1, N, rv, true, pro, uni, Tp);
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch);
    if (!(ok = bar.sync())) break;
    stage_T_norms<VT, NT>(p.Tred, N, sT, s_tn2, scratch);
    // slots: plain CG: s_sig = sum r r_i^2, s_gam = (r, r); preconditioned: s_sig = (r, z)
    // (the CG gamma), s_gam = (r, r) (the stopping rule's norm)
    if (t < NT) {
      const double sg = t < N ? __ldcg(p.Tred + N * N + t) : 0.0;
      const double gm = t < N ? __ldcg(p.Tred + N * N + N + t) : 0.0;
      s_sig[t] = sg;
      s_gam[t] = gm;
      s_bn2[t] = gm;
      s_active[t] = (t < N && !s_done[t] && gm > 0.0) ? 1 : 0;
      s_alpha[t] = 0.0;
      s_beta[t] = 0.0;
      s_spare[t] = 0.0;
    }
    __syncthreads();
    tick(PH_SETUP);
    const int limit = fixed ? p.fixed_iters : (p.max_iter - total_iter);
    int it = 0;
    for (;;) {
      // scalars of this step (identical in every CTA: same sums in the same order)
      if (t < N) {
        int a = s_active[t];
        const double gm = s_gam[t];
        if (a && it > 0) {
          if (!isfinite(gm)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
          else if (fixed ? gm == 0.0 : sqrt(gm) <= s_itol[t] * sqrt(s_bn2[t])) a = 0;
        }
        double al = 0.0, be = 0.0;
        if (a) {
          // CG gamma: (r, r) plain, (r, R^-1 r) preconditioned; delta = (z, S z)
          const double cg = PC ? s_sig[t] : gm;
          const double delta = s_tn2[t] * inv_nm1 + s_sig[t];
          double den = delta;
          if (it > 0) {
            be = cg / s_gold[t];
            den = delta - be * cg / s_alpha[t];
          }
          if (!isfinite(den)) { atomicOr(p.status, DS_NONFINITE); a = 0; be = 0.0; }
          else if (den <= 0.0) { atomicOr(p.status, DS_BREAKDOWN); a = 0; be = 0.0; }
          else al = cg / den;
        }
        s_active[t] = a;
        s_alpha[t] = al;
        s_beta[t] = be;
        s_alpha_v[t] = (VT)al;
        s_beta_v[t] = (VT)be;
      }
      __syncthreads();
      if (t == 0) {
        int any = 0;
        for (int j = 0; j < N; ++j) any |= s_active[j];
        s_flag[0] = any && it < limit;
      }
      __syncthreads();
      if (!s_flag[0]) break;
      tick(PH_SCAL);
      passF<VT, NT, PC>(HA, row0, row1, N, X, Res, P, Sv, rv, sT, s_alpha_v, s_beta_v, (VT)inv_nm1,
                        tiles, Tp);
      tick(PH_PASS);
      if (!(ok = bar.sync())) break;
      tick(PH_BAR1);
      reduce_slice(p.Tpart, G, NE, p.Tred, scratch);
      tick(PH_RED);
      if (!(ok = bar.sync())) break;
      tick(PH_BAR2);
      stage_T_norms<VT, NT>(p.Tred, N, sT, s_tn2, scratch);
      if (t < N) {
        if (s_active[t]) {
          s_iters[t] += 1;
          s_gold[t] = PC ? s_sig[t] : s_gam[t];
          s_gam[t] = __ldcg(p.Tred + N * N + N + t);
          s_sig[t] = __ldcg(p.Tred + N * N + t);
        }
      }
      __syncthreads();
      tick(PH_SCAL);
      ++it;
    }
    if (!ok) break;
    total_iter += it;

    // ---- refresh: Z (+)= X; T = HA^T Z; W = T/(N-1); true residual D - S Z; next right-hand
    // side. FP64 in the FP64 mode; double-float (FP32 pairs) in the FP32 mode.
    if constexpr (sizeof(VT) == 8) {
      ProRefresh<VT> pro{p.Z, X, N, refine};
      passA<double, NT>(p.HA64, row0, row1, N, p.r, false, pro, uni, Tp);
    } else {
      ProRefreshDF<VT> pro{p.Zdf, X, N, true};
      passA<df32, NT>(p.HAdf, row0, row1, N, static_cast<const df32*>(nullptr), false, pro, uni, Tp);
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch);
    if (!(ok = bar.sync())) break;
    if (b == 0)
      for (int e = t; e < N * N; e += kThreads) p.W[e] = __ldcg(p.Tred + e) * inv_nm1;
    if (!refine && !p.true_residual) {
      tick(PH_REFRESH);
      break;
    }
    if constexpr (sizeof(VT) == 8) {
      double* sT64 = reinterpret_cast<double*>(uni);
      stage_T<double, NT>(p.Tred, N, sT64);
      constexpr int LD64 = NT + 2;
      EpiRefresh<VT> epi{p.Z, p.D, p.r, nullptr, inv_nm1, N};
      passB<double, NT>(p.HA64, row0, row1, N, sT64, uni + NT * LD64 * sizeof(double), epi, s_tmp);
    } else {
      df32* sTd = reinterpret_cast<df32*>(uni);
      stage_T<df32, NT>(p.Tred, N, sTd);
      constexpr int LDD = NT + 2;
      EpiRefreshDF<VT> epi{p.Zdf, p.Ddf, p.r, static_cast<VT*>(p.B), N, df32(inv_nm1)};
      passB<df32, NT>(p.HAdf, row0, row1, N, sTd, uni + NT * LDD * sizeof(df32), epi, s_tmp);
    }
    if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
    if (!(ok = bar.sync())) break;
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_tmp, scratch);
    par ^= 1;
    ++refinements;
    if (t < N) {
      const double tr = s_dn2[t] > 0.0 ? sqrt(s_tmp[t] / s_dn2[t]) : 0.0;
      s_true[t] = tr;
      if (refine) {
        if (tr <= p.tol) s_done[t] = 1;
        // next inner solve only has to gain the remaining factor tol/tr (with margin 0.1)
        s_itol[t] = fmax(p.inner_tol, tr > 0.0 ? 0.1 * p.tol / tr : p.inner_tol);
        if (s_itol[t] > 0.5) s_itol[t] = 0.5;
      }
    }
    __syncthreads();
    if (t == 0) {
      int all = 1;
      for (int j = 0; j < N; ++j) all &= s_done[j];
      s_flag[1] = all;
    }
    __syncthreads();
    tick(PH_REFRESH);
    if (!refine || fixed || s_flag[1] || outer >= p.max_refine || total_iter >= p.max_iter) break;
    ++outer;
  }

  if (b == 0) {
    if (t < N) {
      p.col_iters[t] = s_iters[t];
      const double rec = s_dn2[t] > 0.0 ? sqrt(s_gam[t] / s_dn2[t]) : 0.0;
      p.col_relres[t] = refine ? s_true[t] : rec;
      p.col_true[t] = s_true[t];
      bool conv;
      if (fixed) conv = true;
      else if (refine) conv = s_true[t] >= 0.0 && s_true[t] <= p.tol;
      else conv = s_dn2[t] == 0.0 || sqrt(s_gam[t]) <= p.tol * sqrt(s_dn2[t]);
      if (!conv && ok) atomicOr(p.status, DS_NOT_CONVERGED);
    }
    if (t == 0) p.status[1] = refinements;
    if (prof) {
      ph[PH_REFRESH] += 0;
      for (int q = 0; q < PH_COUNT; ++q) p.prof[q] = ph[q];
    }
  }
}

// ------------------------------------------------------------------ K1: innovations
template <typename VT>
__global__ void __launch_bounds__(kThreads) innov_kernel(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ HA64, float* __restrict__ HA32, double* __restrict__ D,
    float* __restrict__ B32, __nv_bfloat16* __restrict__ HAb, __half* __restrict__ HAh,
    int split_lo, df32* __restrict__ HAdf, df32* __restrict__ Ddf) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    double z[4] = {0.0, 0.0, 0.0, 0.0};
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
    double s = z[0] + z[1] + z[2] + z[3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double zbar = s / (double)N;
    const double yi = y[i], sr = sqrt(r[i]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = lane + 32 * q;
      if (j < N) {
        const int64_t e = i * N + j;
        double pert = 0.0;
        if (emode == 1) pert = E[e];
        else if (emode == 2) pert = sr * perturbation_normal(i, j, seed, counter);
        const double ha = z[q] - zbar;
        const double d = (yi - z[q]) + pert;
        HA64[e] = ha;
        D[e] = d;
        if (HA32) HA32[e] = (float)ha;
        if (B32) B32[e] = (float)d;
        if (HAdf) HAdf[e] = df32(ha);
        if (Ddf) Ddf[e] = df32(d);
        // low-precision copies: hi part at [0, m N), lo part (ha - hi) at [m N, 2 m N) when split
        if (HAb) {
          const __nv_bfloat16 hi = __double2bfloat16(ha);
          HAb[e] = hi;
          if (split_lo) HAb[m * N + e] = __double2bfloat16(ha - (double)__bfloat162float(hi));
        }
        if (HAh) {
          const __half hi = __double2half(ha);
          HAh[e] = hi;
          if (split_lo) HAh[m * N + e] = __double2half(ha - (double)__half2float(hi));
        }
      }
    }
  }
}

__global__ void draw_perturbations_kernel(uint64_t seed, uint64_t counter,
                                          const double* __restrict__ r, int64_t m, int N,
                                          double* __restrict__ E) {
  const int64_t total = m * N;
  for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * kThreads) {
    const int64_t i = e / N;
    const int j = (int)(e % N);
    E[e] = sqrt(r[i]) * perturbation_normal(i, j, seed, counter);
  }
}

__global__ void convert_r_kernel(const double* __restrict__ r, float* __restrict__ r32, int64_t m) {
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < m; i += (int64_t)gridDim.x * kThreads)
    r32[i] = (float)r[i];
}

// ------------------------------------------------------------------ K4: final update
// MODE 0: X_a = X_f + (X_f - xbar 1^T) W (CGD-EnKF, Fig. 2 / Algorithm 1);
// MODE 1: X_a = X_f W (CGD-EnKF-Reduced, Algorithm 2 with W = V).
// Row tiles of TRB rows staged in shared memory.
template <typename VT, int NT, int MODE = 0>
__global__ void __launch_bounds__(kThreads) update_kernel(const VT* Xf, VT* Xa,
                                                          const double* __restrict__ W,
                                                          int64_t n, int N) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int LD = NT + 16 / (int)sizeof(VT), TRB = Tile<NT>::TRB, C4 = NT / 4;
  constexpr int NJ = NT / 4;
  VT* sW = reinterpret_cast<VT*>(smem);
  VT* sX = sW + NT * LD;
  VT* smean = sX + TRB * LD;
  const int t = threadIdx.x, tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * 4;
  const bool vec = (N & 3) == 0;
  for (int e = t; e < NT * LD; e += kThreads) {
    const int k = e / LD, j = e % LD;
    sW[e] = (k < N && j < N) ? (VT)W[k * N + j] : VT(0);
  }
  for (int64_t i0 = (int64_t)blockIdx.x * TRB; i0 < n; i0 += (int64_t)gridDim.x * TRB) {
    __syncthreads();
#pragma unroll
    for (int c = t; c < TRB * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      VT a[4] = {VT(0), VT(0), VT(0), VT(0)};
      if (i < n && c0 < N) ld4<VT>(a, Xf + i * N, c0, N, vec);
#pragma unroll
      for (int y = 0; y < 4; ++y) sX[ii * LD + c0 + y] = a[y];
    }
    __syncthreads();
    if (t < TRB) {
      VT s = VT(0);
      for (int k = 0; k < N; ++k) s += sX[t * LD + k];
      smean[t] = s / (VT)N;
    }
    __syncthreads();
    // original X_f fragments for the output (same threads write X_a, so X_a may alias X_f)
    VT xf[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) xf[x][y] = sX[(r0 + x) * LD + j0 + y];
    __syncthreads();
    if (MODE == 0) {
      for (int e = t; e < TRB * NT; e += kThreads) {
        const int ii = e / NT, k = e % NT;
        if (k < N) sX[ii * LD + k] -= smean[ii];
      }
    }
    __syncthreads();
    VT acc[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = VT(0);
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      VT a[4], bv[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) a[x] = sX[(r0 + x) * LD + k];
      load_vec<VT>(bv, sW + k * LD + j0, 4);
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bv[y], acc[x][y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t i = i0 + r0 + x;
      if (i < n && j0 < N) {
        VT o[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) o[y] = MODE == 0 ? xf[x][y] + acc[x][y] : acc[x][y];
        st4<VT>(Xa + i * N, j0, N, vec, o);
      }
    }
  }
}

template <typename VT, int NT> constexpr int update_smem_bytes() {
  constexpr int LD = NT + 16 / (int)sizeof(VT);
  return (NT * LD + Tile<NT>::TRB * LD + Tile<NT>::TRB) * (int)sizeof(VT);
}

// ------------------------------------------------------------------ host launchers
static int pick_nt(int N) { return N <= 32 ? 32 : (N <= 64 ? 64 : 128); }

template <typename VT>
static void* solve_fn(int NT, bool pc) {
  if (pc) {
    if (NT == 32) return (void*)solve_kernel<VT, 32, true>;
    if (NT == 64) return (void*)solve_kernel<VT, 64, true>;
    return (void*)solve_kernel<VT, 128, true>;
  }
  if (NT == 32) return (void*)solve_kernel<VT, 32, false>;
  if (NT == 64) return (void*)solve_kernel<VT, 64, false>;
  return (void*)solve_kernel<VT, 128, false>;
}
template <typename VT>
static size_t solve_smem(int NT) {
  return NT == 32 ? solve_smem_bytes<VT, 32>() : (NT == 64 ? solve_smem_bytes<VT, 64>() : solve_smem_bytes<VT, 128>());
}

cudaError_t plan_solve(enkf_handle_s* h) {
  const int N = h->cfg.N;
  const int NT = pick_nt(N);
  const bool fp64 = h->cfg.precision == ENKF_FP64;
  const bool pc = h->cfg.precondition != 0;
  void* fn = fp64 ? solve_fn<double>(NT, pc) : solve_fn<float>(NT, pc);
  const size_t smem = fp64 ? solve_smem<double>(NT) : solve_smem<float>(NT);
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int max_coresident = occ * h->sms;
  const int64_t min_rows = 32;
  int G = (int)std::min<int64_t>(max_coresident, std::max<int64_t>(1, (h->cfg.m + min_rows - 1) / min_rows));
  if (h->cfg.grid_blocks > 0) G = std::min(h->cfg.grid_blocks, max_coresident);
  h->launch.G = G;
  h->launch.NT = NT;
  h->launch.smem = smem;
  return cudaSuccess;
}

cudaError_t launch_innovations(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                               int emode, uint64_t seed, uint64_t counter) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const int blocks = (int)std::min<int64_t>((c.m + 7) / 8, (int64_t)h->sms * 16);
  const bool fp64 = c.precision == ENKF_FP64;
  if (fp64)
    innov_kernel<double><<<blocks, kThreads, 0, h->stream>>>(
        static_cast<const double*>(Xf), ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter,
        c.m, c.N, ws.HA64, nullptr, ws.D, nullptr, nullptr, nullptr, 0, nullptr, nullptr);
  else
    innov_kernel<float><<<blocks, kThreads, 0, h->stream>>>(
        static_cast<const float*>(Xf), ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter,
        c.m, c.N, ws.HA64, ws.HA32, ws.D, static_cast<float*>(ws.B),
        c.precision == ENKF_BF16_REFINE ? static_cast<__nv_bfloat16*>(ws.HA16) : nullptr,
        c.precision == ENKF_FP16_REFINE ? static_cast<__half*>(ws.HA16) : nullptr,
        c.lowprec_terms != 1 ? 1 : 0, static_cast<df32*>(ws.HAdf), static_cast<df32*>(ws.Ddf));
  return cudaGetLastError();
}

cudaError_t launch_convert_r(enkf_handle_s* h) {
  if (!h->ws.r32) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((h->cfg.m + kThreads - 1) / kThreads, 4096);
  convert_r_kernel<<<blocks, kThreads, 0, h->stream>>>(h->ws.r, h->ws.r32, h->cfg.m);
  return cudaGetLastError();
}

cudaError_t launch_solve(enkf_handle_s* h) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  const bool fp64 = c.precision == ENKF_FP64;
  SolveParams p{};
  p.m = c.m;
  p.N = c.N;
  p.mode = fp64 ? 0 : 1;
  p.HA = fp64 ? (const void*)ws.HA64 : (const void*)ws.HA32;
  p.HA64 = ws.HA64;
  p.D = ws.D;
  p.r = ws.r;
  p.rv = fp64 ? (const void*)ws.r : (const void*)ws.r32;
  p.B = ws.B;
  p.X = ws.X;
  p.Res = ws.Res;
  p.P = ws.P;
  p.Sv = ws.Sv;
  p.Z = ws.Z;
  p.HAdf = static_cast<const df32*>(ws.HAdf);
  p.Ddf = static_cast<const df32*>(ws.Ddf);
  p.Zdf = static_cast<df32*>(ws.Zdf);
  p.Tpart = ws.Tpart;
  p.Tred = ws.Tred;
  p.rrpart = ws.rrpart;
  p.W = ws.W;
  p.prof = h->prof_enabled ? ws.prof : nullptr;
  p.tol = c.tol;
  p.inner_tol = c.inner_tol;
  p.max_iter = c.max_iter;
  p.fixed_iters = c.fixed_iters;
  p.max_refine = c.max_refine;
  p.true_residual = c.true_residual;
  p.col_iters = ws.col_iters;
  p.col_relres = ws.col_relres;
  p.col_true = ws.col_true;
  p.status = ws.status;
  p.bar = ws.bar;
  cudaError_t err = cudaMemsetAsync(ws.bar, 0, 4 * sizeof(unsigned), h->stream);
  if (err != cudaSuccess) return err;
  err = cudaMemsetAsync(ws.status, 0, 4 * sizeof(int32_t), h->stream);
  if (err != cudaSuccess) return err;
  const bool pc = c.precondition != 0;
  void* fn = fp64 ? solve_fn<double>(h->launch.NT, pc) : solve_fn<float>(h->launch.NT, pc);
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel(fn, dim3(h->launch.G), dim3(kThreads), args,
                                     h->launch.smem, h->stream);
}

template <int MODE>
static cudaError_t launch_update_mode(enkf_handle_s* h, const void* Xf, void* Xa) {
  const auto& c = h->cfg;
  const int NT = h->launch.NT;
  const bool fp64 = c.precision == ENKF_FP64;
  const int TRB = NT == 32 ? Tile<32>::TRB : (NT == 64 ? Tile<64>::TRB : Tile<128>::TRB);
  const int tiles = (int)std::min<int64_t>((c.n + TRB - 1) / TRB, (int64_t)h->sms * 8);
  void* fn;
  int smem;
  if (fp64) {
    fn = NT == 32 ? (void*)update_kernel<double, 32, MODE> : NT == 64 ? (void*)update_kernel<double, 64, MODE> : (void*)update_kernel<double, 128, MODE>;
    smem = NT == 32 ? update_smem_bytes<double, 32>() : NT == 64 ? update_smem_bytes<double, 64>() : update_smem_bytes<double, 128>();
  } else {
    fn = NT == 32 ? (void*)update_kernel<float, 32, MODE> : NT == 64 ? (void*)update_kernel<float, 64, MODE> : (void*)update_kernel<float, 128, MODE>;
    smem = NT == 32 ? update_smem_bytes<float, 32>() : NT == 64 ? update_smem_bytes<float, 64>() : update_smem_bytes<float, 128>();
  }
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (err != cudaSuccess) return err;
  const double* W = h->ws.W;
  int64_t n = c.n;
  int N = c.N;
  void* args[] = {const_cast<void**>(&Xf), &Xa, const_cast<double**>(&W), &n, &N};
  return cudaLaunchKernel(fn, dim3(tiles), dim3(kThreads), args, smem, h->stream);
}

cudaError_t launch_update(enkf_handle_s* h, const void* Xf, void* Xa) {
  return launch_update_mode<0>(h, Xf, Xa);
}

cudaError_t launch_update_product(enkf_handle_s* h, const void* Xf, void* Xa) {
  return launch_update_mode<1>(h, Xf, Xa);
}

cudaError_t launch_draw_perturbations(uint64_t seed, uint64_t counter, const double* r, int64_t m,
                                      int N, double* E, cudaStream_t s) {
  const int64_t total = m * N;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + kThreads - 1) / kThreads, 4096));
  draw_perturbations_kernel<<<blocks, kThreads, 0, s>>>(seed, counter, r, m, N, E);
  return cudaGetLastError();
}

}  // namespace enkf
