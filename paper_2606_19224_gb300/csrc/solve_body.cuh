// The persistent CG solve of one problem by a set of co-resident CTAs, and the row-range
// form of the update step: shared by the single-analysis kernels (kernels_fp.cu) and the
// batched kernel (kernels_batch.cu). The innovations are in innov_device.cuh.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cg_device.cuh"

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
  int warm;                  // FP32 mode: Zdf holds a starting solution (learned warm start)
  int warm_accept;           // 1: keep every finite start; 0: only those with ||B_j|| <= ||d_j||
  double* Tacc = nullptr;    // FP32 mode, atomic_reduce: [3][N N + 4 N] rotating step totals
  int atomic_reduce = 0;     // FP32 mode: a step's sums are added into Tacc (one barrier per step)
  double* col_warm;          // [N] relative residual ||B_j|| / ||d_j|| of that start
};


// The persistent solve of one problem by G co-resident CTAs (this one is number b), with the
// grid barrier `bar` over exactly those CTAs: the whole grid for one analysis, a team of the
// grid for batched analyses.
template <typename VT, int NT, bool PC>
__device__ void solve_body(const SolveParams& p, const int G, const int b, GridBarrier& bar,
                           unsigned char* smem) {
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
  double* s_den = s_true + NT;
  int* s_active = reinterpret_cast<int*>(s_den + NT);
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

  const int N = p.N, t = threadIdx.x;
  // every CTA of the launch sees the same size, so all of them leave here together
  if (dynamic_smem_bytes() < (unsigned)solve_smem_bytes<VT, NT>()) {
    if (t == 0) atomicOr(p.status, DS_SMEM);
    return;
  }
  const int64_t rows_per = (p.m + G - 1) / G;
  const int64_t row0 = imin64(p.m, (int64_t)b * rows_per);
  const int64_t row1 = imin64(p.m, row0 + rows_per);
  const int NE = N * N + 4 * N;   // [N x N Gram | four N-vectors of column sums]
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
  // atomic_reduce (FP32 mode): CG steps so far (the same in every CTA) pick the step's
  // accumulator; all three start at zero (ordered before their first use by the first barrier)
  const bool atomic = sizeof(VT) == 4 && p.atomic_reduce && p.Tacc != nullptr;
  int gstep = 0;
  if (atomic) {
    const int chunk = (3 * NE + G - 1) / G;
    const int e1 = min(3 * NE, (b + 1) * chunk);
    for (int e = b * chunk + t; e < e1; e += kThreads) p.Tacc[e] = 0.0;
  }
  // the last two column-sum vectors of the partials are written only by the FP32 step
  if (t < N) {
    Tp[N * N + 2 * N + t] = 0.0;
    Tp[N * N + 3 * N + t] = 0.0;
  }

  // a warm start keeps the given Zdf; B holds its residual (written by the decoder)
  const bool warm = refine && p.warm != 0;
  // ---- ||d_j||^2 (and Z = 0 for the refinement accumulator)
  rows_reduce<NT>(row0, row1, N, [&](int64_t i, int j, double& acc) {
    const double d = p.D[i * N + j];
    acc = fma(d, d, acc);
    if (refine && !warm) p.Zdf[i * N + j] = df32(0.f, 0.f);
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
  if (ok && warm) {
    // the start's true residual judges it: a column whose start is non-finite or (unless
    // warm_accept) whose residual is larger than the zero start's (d_j) falls back to
    // z_j = 0, B_j = d_j
    VT* Bv = static_cast<VT*>(p.B);
    rows_reduce<NT>(row0, row1, N, [&](int64_t i, int j, double& acc) {
      const double v = (double)Bv[i * N + j];
      acc = fma(v, v, acc);
    }, s_tmp, scratch);
    if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
    ok = bar.sync();
    if (ok) {
      reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_tmp, scratch);
      par ^= 1;
      if (t < NT) {
        const bool bad = t < N && !s_done[t] &&
                         (p.warm_accept ? !isfinite(s_tmp[t]) : !(s_tmp[t] <= s_dn2[t]));
        if (b == 0 && t < N) p.col_warm[t] = s_dn2[t] > 0.0 ? sqrt(s_tmp[t] / s_dn2[t]) : 0.0;
        s_active[t] = bad ? 1 : 0;   // s_active is free until the first inner solve
        if (t < N && !s_done[t] && !bad) {
          const double tr = sqrt(s_tmp[t] / s_dn2[t]);
          s_itol[t] = fmin(0.5, fmax(p.inner_tol, tr > 0.0 ? 0.1 * p.tol / tr : p.inner_tol));
        }
      }
      __syncthreads();
      int nbad = 0;
      for (int j = 0; j < N; ++j) nbad += s_active[j];
      if (nbad) {
        for (int64_t e = (int64_t)t; e < (row1 - row0) * N; e += kThreads) {
          const int64_t i = row0 + e / N;
          const int j = (int)(e % N);
          if (s_active[j]) {
            p.Zdf[i * N + j] = df32(0.f, 0.f);
            Bv[i * N + j] = (VT)p.D[i * N + j];
          }
        }
        if (b == 0 && t == 0) p.status[2] = nbad;
      }
      __syncthreads();
    }
  }
  tick(PH_SETUP);

  // the CG steps read T only as the staged CT copy: FP32 modes take it from an FP32 T
  const int t_f32 = sizeof(VT) == 4 ? N * N : 0;
  int outer = 0, total_iter = 0, refinements = 0;
  while (ok) {
   if constexpr (sizeof(VT) == 4) {
    // ---- FP32 inner solve of S X = B from X = 0 in the one-reduction Hestenes-Stiefel form
    // (passH): the first reduction gives [HA^T z_0 | sum r_i z_0^2 | (r_0, r_0)], T_0 = HA^T z_0
    {
      ProSetup<VT, PC> pro{B, X, Res, rv, N};
      passA<VT, NT, ProSetup<VT, PC>, PC>(HA, row0, row1, N, rv, true, pro, uni, Tp);
    }
    if (t < N) {
      Tp[N * N + 2 * N + t] = 0.0;
      Tp[N * N + 3 * N + t] = 0.0;
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, t_f32);
    if (!(ok = bar.sync())) break;
    float* sTf = reinterpret_cast<float*>(sT);
    float* bvf = reinterpret_cast<float*>(s_beta_v);
    float* avf = reinterpret_cast<float*>(s_alpha_v);
    if (t < NT) bvf[t] = 0.f;
    __syncthreads();
    stage_T_rec<NT>(p.Tred, N, bvf, sTf, s_tn2, scratch);
    // slots: s_sig = gamma = (r, z); s_den = sum r_i p^2; s_gam = (r, r), the stopping rule's norm
    if (t < NT) {
      const double sg = t < N ? __ldcg(p.Tred + N * N + t) : 0.0;       // sum r_i z_0^2
      const double gm = t < N ? __ldcg(p.Tred + N * N + N + t) : 0.0;   // (r_0, r_0)
      s_sig[t] = PC ? sg : gm;
      s_den[t] = sg;
      s_gam[t] = gm;
      s_bn2[t] = gm;
      s_active[t] = (t < N && !s_done[t] && gm > 0.0) ? 1 : 0;
    }
    __syncthreads();
    tick(PH_SETUP);
    const int limit = fixed ? p.fixed_iters : (p.max_iter - total_iter);
    int it = 0;
    for (;;) {
      // alpha_k = gamma_k / (p_k, S p_k), (p, S p) = ||T_k||^2/(N-1) + sum r_i p^2 (identical in
      // every CTA: same sums in the same order)
      int my_active = 0;
      if (t < N) {
        int a = s_active[t];
        const double gm = s_gam[t];
        if (a && it > 0) {
          const double itm = s_itol[t] * (1.0 - 4.0 * 2.220446049250313e-16);
          if (!isfinite(gm)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
          else if (fixed ? gm == 0.0 : gm <= itm * itm * s_bn2[t]) a = 0;
        }
        double al = 0.0;
        if (a) {
          const double pq = s_tn2[t] * inv_nm1 + s_den[t];
          if (!isfinite(pq)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
          else if (pq <= 0.0) { atomicOr(p.status, DS_BREAKDOWN); a = 0; }
          else al = s_sig[t] / pq;
        }
        s_active[t] = a;
        avf[t] = (float)al;
        my_active = a;
      }
      if (!(__syncthreads_or(my_active) && it < limit)) break;
      tick(PH_SCAL);
      // the step's sums: into this CTA's partial (then a fixed-order reduction between two grid
      // barriers), or added into the step's accumulator (atomic_reduce: one barrier; the
      // accumulator two steps ahead is cleared behind it, every CTA having read it before)
      double* acc = atomic ? p.Tacc + (size_t)(gstep % 3) * NE : Tp;
      if ((N & 3) == 0)
        passH<NT, PC, true>(reinterpret_cast<const float*>(HA), row0, row1, N, reinterpret_cast<float*>(X),
                            reinterpret_cast<float*>(Res), reinterpret_cast<float*>(P),
                            reinterpret_cast<const float*>(rv), sTf, avf, bvf, (float)inv_nm1, tiles, acc,
                            atomic);
      else
        passH<NT, PC, false>(reinterpret_cast<const float*>(HA), row0, row1, N, reinterpret_cast<float*>(X),
                             reinterpret_cast<float*>(Res), reinterpret_cast<float*>(P),
                             reinterpret_cast<const float*>(rv), sTf, avf, bvf, (float)inv_nm1, tiles, acc,
                             atomic);
      tick(PH_PASS);
      if (!(ok = bar.sync())) break;
      tick(PH_BAR1);
      const double* tsum = p.Tred;
      if (atomic) {
        double* z = p.Tacc + (size_t)((gstep + 2) % 3) * NE;
        const int chunk = (NE + G - 1) / G;
        const int e1 = min(NE, (b + 1) * chunk);
        for (int e = b * chunk + t; e < e1; e += kThreads) z[e] = 0.0;
        tsum = acc;
        ++gstep;
      } else {
        reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, t_f32);
        tick(PH_RED);
        if (!(ok = bar.sync())) break;
        tick(PH_BAR2);
      }
      // beta_k = gamma_{k+1} / gamma_k, T_{k+1} = HA^T z_{k+1} + beta_k T_k, sum r_i p_{k+1}^2
      // from the expanded sums; frozen columns keep beta = 0 (their next p is never used:
      // alpha = 0)
      stage_T_rec<NT>(tsum, N, bvf, sTf, s_tn2, scratch, true, s_active, s_sig, s_den, s_gam, s_iters);
      tick(PH_SCAL);
      ++it;
    }
    if (!ok) break;
    total_iter += it;
   } else {
    // ---- inner solve of S X = B from X = 0: first reduction of [HA^T r | sum r_i r^2 | (r, r)]
    {
      ProSetup<VT, PC> pro{B, X, Res, rv, N};
      passA<VT, NT, ProSetup<VT, PC>, PC>(HA, row0, row1, N, rv, true, pro, uni, Tp);
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, t_f32);
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
      s_den[t] = 0.0;
    }
    __syncthreads();
    tick(PH_SETUP);
    const int limit = fixed ? p.fixed_iters : (p.max_iter - total_iter);
    int it = 0;
    for (;;) {
      // scalars of this step (identical in every CTA: same sums in the same order)
      int my_active = 0;
      if (t < N) {
        int a = s_active[t];
        const double gm = s_gam[t];
        if (a && it > 0) {
          // |r| <= itol |b| in squares (itol shrunk by 4 ulps: a stop implies the square-root
          // form); FP64 square roots and divisions are costly on this part's FP64 pipe
          const double itm = s_itol[t] * (1.0 - 4.0 * 2.220446049250313e-16);
          if (!isfinite(gm)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
          else if (fixed ? gm == 0.0 : gm <= itm * itm * s_bn2[t]) a = 0;
        }
        double al = 0.0, be = 0.0;
        if (a) {
          // CG gamma: (r, r) plain, (r, R^-1 r) preconditioned; delta = (z, S z). With
          // beta = gamma / gamma_prev and alpha_prev = gamma_prev / den_prev, the
          // Chronopoulos-Gear denominator delta - beta gamma / alpha_prev is
          // delta - beta^2 den_prev: one division fewer per step.
          const double cg = PC ? s_sig[t] : gm;
          const double delta = s_tn2[t] * inv_nm1 + s_sig[t];
          double den = delta;
          if (it > 0) {
            be = cg / s_gold[t];
            den = delta - be * be * s_den[t];
          }
          if (!isfinite(den)) { atomicOr(p.status, DS_NONFINITE); a = 0; be = 0.0; }
          else if (den <= 0.0) { atomicOr(p.status, DS_BREAKDOWN); a = 0; be = 0.0; }
          else al = cg / den;
          s_den[t] = den;   // den_prev of the next step
        }
        s_active[t] = a;
        s_alpha[t] = al;
        s_beta[t] = be;
        s_alpha_v[t] = (VT)al;
        s_beta_v[t] = (VT)be;
        my_active = a;
      }
      if (!(__syncthreads_or(my_active) && it < limit)) break;
      tick(PH_SCAL);
      if constexpr (async_passF<VT, NT>()) {
        if ((N & 3) == 0)
          passF_async<NT, PC>(HA, row0, row1, N, X, Res, P, Sv, rv, sT, s_alpha_v, s_beta_v, (VT)inv_nm1,
                              tiles, Tp);
        else
          passF<VT, NT, PC>(HA, row0, row1, N, X, Res, P, Sv, rv, sT, s_alpha_v, s_beta_v, (VT)inv_nm1,
                            tiles, Tp);
      } else {
        passF<VT, NT, PC>(HA, row0, row1, N, X, Res, P, Sv, rv, sT, s_alpha_v, s_beta_v, (VT)inv_nm1,
                          tiles, Tp);
      }
      tick(PH_PASS);
      if (!(ok = bar.sync())) break;
      tick(PH_BAR1);
      reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, t_f32);
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
   }

    // ---- refresh: Z (+)= X; T = HA^T Z; W = T/(N-1); true residual D - S Z; next right-hand
    // side. FP64 in the FP64 mode; double-float (FP32 pairs) in the FP32 mode.
    if constexpr (sizeof(VT) == 8) {
      ProRefresh<VT> pro{p.Z, X, N, refine};
      passA<double, NT>(p.HA64, row0, row1, N, p.r, false, pro, uni, Tp);
    } else {
      if ((N & 3) == 0) {
        refreshA_async<NT>(p.HAdf, p.Zdf, reinterpret_cast<const float*>(X), row0, row1, N, uni, Tp);
      } else {
        ProRefreshDF<VT> pro{p.Zdf, X, N, true};
        passA<df32, NT>(p.HAdf, row0, row1, N, static_cast<const df32*>(nullptr), false, pro, uni, Tp);
      }
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b);
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
      bool done_b = false;
      if constexpr (DFTile<NT>::B_ASYNC) {
        if ((N & 3) == 0) {
          refreshB_async<NT, VT>(p.HAdf, p.Zdf, p.Ddf, p.r, static_cast<VT*>(p.B), row0, row1, N, sTd,
                                 df32(inv_nm1), uni + NT * LDD * sizeof(df32), s_tmp);
          done_b = true;
        }
      }
      if (!done_b) {
        EpiRefreshDF<VT> epi{p.Zdf, p.Ddf, p.r, static_cast<VT*>(p.B), N, df32(inv_nm1)};
        passB<df32, NT>(p.HAdf, row0, row1, N, sTd, uni + NT * LDD * sizeof(df32), epi, s_tmp);
      }
    }
    if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
    if (!(ok = bar.sync())) break;
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_tmp, scratch);
    par ^= 1;
    ++refinements;
    if (t < N) {
      // a non-finite residual or ||d_j|| (NaN or Inf in the inputs) ends the column with the
      // non-finite status
      const bool fin = isfinite(s_dn2[t]) && isfinite(s_tmp[t]);
      if (!fin) atomicOr(p.status, DS_NONFINITE);
      const double tr = !fin ? (double)NAN : (s_dn2[t] > 0.0 ? sqrt(s_tmp[t] / s_dn2[t]) : 0.0);
      s_true[t] = tr;
      if (!fin) s_done[t] = 1;
      if (refine) {
        if (tr <= p.tol) s_done[t] = 1;
        // next inner solve only has to gain the remaining factor tol/tr (with margin 0.1)
        s_itol[t] = fmax(p.inner_tol, tr > 0.0 ? 0.1 * p.tol / tr : p.inner_tol);
        if (s_itol[t] > 0.5) s_itol[t] = 0.5;
      }
    }
    const int all_done = __syncthreads_and(t >= N || s_done[t]);
    tick(PH_REFRESH);
    if (!refine || fixed || all_done || outer >= p.max_refine || total_iter >= p.max_iter) break;
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

// ------------------------------------------------------------------ K4: final update
// MODE 0: X_a = X_f + (X_f - xbar 1^T) W (CGD-EnKF, Fig. 2 / Algorithm 1);
// MODE 1: X_a = X_f W (CGD-EnKF-Reduced, Algorithm 2 with W = V).
// Row tiles of TRB rows staged in shared memory.
// Row tiles tile0, tile0 + tstride, ... (TRB rows each) of the update.
template <typename VT, int NT, int MODE = 0>
__device__ __forceinline__ void update_rows(const VT* Xf, VT* Xa, const double* __restrict__ W,
                                            int64_t n, int N, int64_t tile0, int64_t tstride,
                                            unsigned char* smem) {
  constexpr int LD = NT + 16 / (int)sizeof(VT), TRB = Tile<NT>::TRB, C4 = NT / 4;
  constexpr int NJ = NT / 4;
  VT* sW = reinterpret_cast<VT*>(smem);
  VT* sXb[2] = {sW + NT * LD, sW + NT * LD + TRB * LD};   // X_f row tiles, double-buffered
  VT* smean = sW + NT * LD + 2 * TRB * LD;
  const int t = threadIdx.x, tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * 4;
  const bool vec = (N & 3) == 0;
  for (int e = t; e < NT * LD; e += kThreads) {
    const int k = e / LD, j = e % LD;
    sW[e] = (k < N && j < N) ? (VT)__ldcg(W + k * N + j) : VT(0);   // W may be written by this launch
  }
  // the tile of rows [i0, i0 + TRB) into dst: 16-byte cp.async pieces (zero-filled past n and
  // N) when rows are 16-byte aligned (N % 4 == 0), else plain loads
  auto load_tile = [&](int64_t i0, VT* dst) {
#pragma unroll
    for (int c = t; c < TRB * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      const bool ok = i < n && c0 < N;
      if (vec) {
        const VT* src = ok ? Xf + i * N + c0 : Xf;
#pragma unroll
        for (int q = 0; q < (int)sizeof(VT) / 4; ++q)
          cp_async16(dst + ii * LD + c0 + q * (16 / (int)sizeof(VT)), src + q * (16 / (int)sizeof(VT)), ok);
      } else {
        VT a[4] = {VT(0), VT(0), VT(0), VT(0)};
        if (ok) ld4<VT>(a, Xf + i * N, c0, N, false);
#pragma unroll
        for (int y = 0; y < 4; ++y) dst[ii * LD + c0 + y] = a[y];
      }
    }
  };
  int cur = 0;
  if (vec && tile0 * TRB < n) load_tile(tile0 * TRB, sXb[0]);
  cp_async_commit();
  for (int64_t i0 = tile0 * TRB; i0 < n; i0 += tstride * TRB) {
    VT* sX = sXb[cur];
    const int64_t inext = i0 + tstride * TRB;
    if (vec) {
      if (inext < n) load_tile(inext, sXb[cur ^ 1]);   // overlaps this tile's work
      cp_async_commit();
      cp_async_wait<1>();                               // this tile has landed
    } else {
      load_tile(i0, sX);
    }
    __syncthreads();
    // row means: four threads per row (consecutive rows on consecutive lane groups read
    // distinct banks), partial sums over k = g, g + 4, ..., added by two shuffle steps
    for (int rr = t / 4; rr < TRB; rr += kThreads / 4) {
      VT sm = VT(0);
      for (int k = t % 4; k < N; k += 4) sm += sX[rr * LD + k];
      sm += __shfl_xor_sync(0xffffffffu, sm, 1);
      sm += __shfl_xor_sync(0xffffffffu, sm, 2);
      if ((t & 3) == 0) smean[rr] = sm / (VT)N;
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
    __syncthreads();   // every read of sX ends before the next iteration refills it
    cur ^= 1;
  }
  cp_async_wait<0>();
}

template <typename VT, int NT> __host__ __device__ constexpr int update_smem_bytes() {
  constexpr int LD = NT + 16 / (int)sizeof(VT);
  return (NT * LD + 2 * Tile<NT>::TRB * LD + Tile<NT>::TRB) * (int)sizeof(VT);
}

}  // namespace enkf
