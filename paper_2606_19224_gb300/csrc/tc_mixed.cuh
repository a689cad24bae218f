// Mixed-precision CGD-EnKF solve on the 5th-generation tensor cores (tcgen05, TMEM).
//
// The two contractions of every CG step (Eq. matvec_decomp) run as BF16 or FP16 MMAs with
// FP32 accumulation in tensor memory; vectors are FP32; the CG scalars are FP64:
//   u = HA T / (N-1)          one M=128 x N x K=N MMA per 128-row tile (D in TMEM)
//   T_next = HA^T z_next      one M=128 (k, zero-padded) x N x K=128 MMA per tile,
//                             accumulated in TMEM across the CTA's tiles
// Each inner CG solve (for a correction, from zero) runs until its residual fell by a
// precision-dependent factor (or for at most `refresh_every` steps); then the correction is
// added to the solution, kept in double-float (FP32 pairs), and the true residual D - S Z is
// recomputed in double-float on CUDA cores as the next inner right-hand side (iterative
// refinement of the low-precision solve, with an FP64-grade final residual check).
//
// Operands are staged by this kernel into shared memory in the canonical K-major,
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix, K-direction core stride
// 128 B = descriptor LBO, row-group stride = descriptor SBO). One thread issues the MMAs;
// completion is signalled through an mbarrier by tcgen05.commit; every wait is bounded.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "cg_device.cuh"

namespace enkf {

// ------------------------------------------------------------------ tcgen05 / mbarrier PTX
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of tcgen05; no swizzle, base offset 0
  return d;
}
// kind::f16 instruction descriptor: D F32, A = B = F16 (fmt 0) or BF16 (fmt 1), both
// K-major, dense, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar)));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}
// bounded wait for the given phase; returns false (and raises DS_TIMEOUT) if it never completes
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase, int* status) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  while (!done) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_addr(mbar)), "r"(phase));
    if (!done && global_ns() - t0 > kBarrierTimeoutNs) {
      atomicOr(status, DS_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

template <typename T16> struct H16;
template <> struct H16<__nv_bfloat16> {
  static constexpr uint32_t fmt = 1;
  __device__ static __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
};
template <> struct H16<__half> {
  static constexpr uint32_t fmt = 0;
  __device__ static __half from(float x) { return __float2half_rn(x); }
};

// element (r, k) of a K-major operand with Kd K-elements per row, in elements of 2 bytes:
// core matrix (r/8, k/8) at ((r/8)*(Kd/8) + k/8) * 64, then (r%8)*8 + k%8
__device__ __forceinline__ int core_idx(int r, int k, int Kd) {
  return (((r >> 3) * (Kd >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

constexpr int kTR = 128;  // rows per tile = M of the u MMA = K of the Gram MMA

template <int NT> __host__ __device__ constexpr int tc_tmem_cols() { return (2 * NT) < 32 ? 32 : 2 * NT; }
template <int NT, int TERMS> __host__ __device__ constexpr int tc_bytes() {
  // sAu [128][NT] (reused as sBg [NT][128] once the u MMA has consumed it), sBu [NT][NT],
  // sAg [128][128] (2-byte; hi and lo copies when the operands are split), sacc [8][2][NT] f32,
  // scales zs, ts [NT] f32
  return (TERMS == 3 ? 2 : 1) * 2 * (kTR * NT + NT * NT + kTR * kTR) + 4 * (8 * 2 * NT) + 4 * 2 * NT;
}

// ------------------------------------------------------------------ fused tensor-core CG step
// Same recurrences as passF (Chronopoulos-Gear arrangement, optionally preconditioned by R);
// the contractions run on the tensor cores. sBu holds (T/(N-1)) scaled per column by ts_j,
// the Gram operand holds z scaled per column by zs_j (so FP16 neither overflows nor flushes);
// the scales are undone on the FP32 values read from TMEM.
//
// TERMS == 3: every operand is split into x_hi = round(x) and x_lo = round(x - x_hi) and each
// product is formed as hi*hi + hi*lo + lo*hi (three MMAs into the same accumulator), about 16
// significant bits instead of 8 (BF16) or 11 (FP16). Tiles: [hi | lo] pairs of each operand.
template <typename T16, int NT, bool PC, int TERMS>
__device__ void passF_tc(const T16* __restrict__ HAhi, const T16* __restrict__ HAlo, int64_t row0,
                         int64_t row1, int N, float* X, float* Res, float* P, float* Sv,
                         const float* __restrict__ rv, const float* alpha, const float* beta,
                         const float* zs, const float* ts, T16* sAu, const T16* sBu, T16* sAg,
                         T16* sBg, float* sacc, uint32_t tmem, uint64_t* mbar_u, uint64_t* mbar_g,
                         uint32_t& ph_u, uint32_t& ph_g, int* status, bool& ok,
                         double* __restrict__ out) {
  constexpr bool SPLIT = TERMS == 3;
  constexpr uint32_t idesc = umma_idesc(H16<T16>::fmt, NT);
  constexpr int HALF = NT / 2, CH = HALF / 16;  // columns per warpgroup, 16-column chunks
  constexpr int AU = kTR * NT, BU = NT * NT, AG = kTR * kTR, BG = NT * kTR;  // tile sizes
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int q = warp & 3, half = warp >> 2;
  const int rt = 32 * q + lane;                 // the thread's row within the tile (TMEM lane)
  const bool vec = (N & 3) == 0;
  const uint32_t d_u = tmem, d_g = tmem + NT;
  for (int e = t; e < 8 * 2 * NT; e += kThreads) sacc[e] = 0.f;
  __syncthreads();
  bool first_tile = true;
  for (int64_t i0 = row0; i0 < row1 && ok; i0 += kTR) {
    // stage HA rows [i0, i0+128): sAu (rows x k, K-major over k) and sAg (k x rows, K-major
    // over rows); zero beyond row1 and beyond N
    for (int c = t; c < kTR * (NT / 8); c += kThreads) {
      const int r = c / (NT / 8), k0 = (c % (NT / 8)) * 8;
      const int64_t i = i0 + r;
#pragma unroll
      for (int part = 0; part < (SPLIT ? 2 : 1); ++part) {
        const T16* src = part ? HAlo : HAhi;
        alignas(16) T16 v[8];
        if (i < row1 && k0 + 8 <= N && ((N & 7) == 0)) {
          *reinterpret_cast<uint4*>(v) = *reinterpret_cast<const uint4*>(src + i * N + k0);
        } else {
#pragma unroll
          for (int y = 0; y < 8; ++y) v[y] = (i < row1 && k0 + y < N) ? src[i * N + k0 + y] : H16<T16>::from(0.f);
        }
        *reinterpret_cast<uint4*>(sAu + part * AU + core_idx(r, k0, NT)) = *reinterpret_cast<const uint4*>(v);
#pragma unroll
        for (int y = 0; y < 8; ++y) sAg[part * AG + core_idx(k0 + y, r, kTR)] = v[y];
      }
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      constexpr uint32_t sbo_u = (NT / 8) * 128;
      const uint32_t au = smem_addr(sAu), bu = smem_addr(sBu);
#pragma unroll
      for (int kb = 0; kb < NT / 16; ++kb) {
        umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc, kb > 0 ? 1u : 0u);
        if (SPLIT) {
          umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + 2 * BU + kb * 256, 128, sbo_u), idesc, 1u);
          umma_f16(d_u, umma_desc(au + 2 * AU + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc, 1u);
        }
      }
      umma_commit(mbar_u);
    }
    const int64_t i = i0 + rt;
    const bool valid = i < row1;
    const float ri = valid ? rv[i] : 1.f;
    const float rinv = 1.f / ri;
    if (!mbar_wait(mbar_u, ph_u, status)) ok = false;
    ph_u ^= 1u;
    tc_fence_after();
    float gA[CH][16], gB[CH][16];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j0 = half * HALF + 16 * c;
      float u[16];
      tmem_ld16(d_u + ((uint32_t)(32 * q) << 16) + j0, u);
#pragma unroll
      for (int y4 = 0; y4 < 4; ++y4) {
        const int jj = j0 + 4 * y4;
        float rr[4] = {0.f, 0.f, 0.f, 0.f}, pp[4] = {0.f, 0.f, 0.f, 0.f};
        float ss[4] = {0.f, 0.f, 0.f, 0.f}, xx[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid && jj < N) {
          ld4<float>(rr, Res + i * N, jj, N, vec);
          ld4<float>(pp, P + i * N, jj, N, vec);
          ld4<float>(ss, Sv + i * N, jj, N, vec);
          ld4<float>(xx, X + i * N, jj, N, vec);
        }
        float pn[4], sn[4], xn[4], rn[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int j = jj + y;
          const float uu = u[4 * y4 + y] / ts[j];
          const float zz = PC ? rr[y] * rinv : rr[y];
          const float ww = PC ? uu + rr[y] : fmaf(ri, rr[y], uu);
          const float be = beta[j], al = alpha[j];
          pn[y] = be == 0.f ? zz : fmaf(be, pp[y], zz);
          sn[y] = be == 0.f ? ww : fmaf(be, ss[y], ww);
          xn[y] = fmaf(al, pn[y], xx[y]);
          rn[y] = fmaf(-al, sn[y], rr[y]);
          const float zn = PC ? rn[y] * rinv : rn[y];
          const bool live = valid && j < N;
          gA[c][4 * y4 + y] = live ? (PC ? rn[y] * zn : ri * rn[y] * rn[y]) : 0.f;
          gB[c][4 * y4 + y] = live ? rn[y] * rn[y] : 0.f;
          const float zsc = live ? zn * zs[j] : 0.f;
          const T16 zh = H16<T16>::from(zsc);
          sBg[core_idx(j, rt, kTR)] = zh;
          if (SPLIT) sBg[BG + core_idx(j, rt, kTR)] = H16<T16>::from(zsc - (float)zh);
        }
        if (valid && jj < N) {
          st4<float>(P + i * N, jj, N, vec, pn);
          st4<float>(Sv + i * N, jj, N, vec, sn);
          st4<float>(X + i * N, jj, N, vec, xn);
          st4<float>(Res + i * N, jj, N, vec, rn);
        }
      }
    }
    // per-column sums over the warp's 32 rows, accumulated in this warp's shared slot
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        float a = gA[c][y], b = gB[c][y];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
          const int j = half * HALF + 16 * c + y;
          sacc[(warp * 2 + 0) * NT + j] += a;
          sacc[(warp * 2 + 1) * NT + j] += b;
        }
      }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      constexpr uint32_t sbo_g = (kTR / 8) * 128;
      const uint32_t ag = smem_addr(sAg), bg = smem_addr(sBg);
#pragma unroll
      for (int kb = 0; kb < kTR / 16; ++kb) {
        umma_f16(d_g, umma_desc(ag + kb * 256, 128, sbo_g), umma_desc(bg + kb * 256, 128, sbo_g), idesc,
                 (first_tile && kb == 0) ? 0u : 1u);
        if (SPLIT) {
          umma_f16(d_g, umma_desc(ag + kb * 256, 128, sbo_g), umma_desc(bg + 2 * BG + kb * 256, 128, sbo_g), idesc, 1u);
          umma_f16(d_g, umma_desc(ag + 2 * AG + kb * 256, 128, sbo_g), umma_desc(bg + kb * 256, 128, sbo_g), idesc, 1u);
        }
      }
      umma_commit(mbar_g);
    }
    // the Gram MMA reads sAg / sBg: wait before the next tile restages them
    if (!mbar_wait(mbar_g, ph_g, status)) ok = false;
    ph_g ^= 1u;
    tc_fence_after();
    first_tile = false;
  }
  // partial Gram from TMEM: thread (lane row k = rt, warpgroup half) -> out[k*N + j] / zs_j
  // (tcgen05.ld is warp-collective: the condition below is uniform within a warp)
  if (!first_tile && 32 * q < N) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j0 = half * HALF + 16 * c;
      float v[16];
      tmem_ld16(d_g + ((uint32_t)(32 * q) << 16) + j0, v);
      if (rt < N) {
#pragma unroll
        for (int y = 0; y < 16; ++y)
          if (j0 + y < N) out[rt * N + j0 + y] = (double)(v[y] / zs[j0 + y]);
      }
    }
  } else if (first_tile) {
    for (int e = t; e < N * N; e += kThreads) out[e] = 0.0;
  }
  tc_fence_before();
  __syncthreads();
  if (t < N) {
    const int h = t / HALF;
    double a = 0.0, b = 0.0;
    for (int w = 4 * h; w < 4 * h + 4; ++w) {
      a += (double)sacc[(w * 2 + 0) * NT + t];
      b += (double)sacc[(w * 2 + 1) * NT + t];
    }
    out[N * N + t] = a;
    out[N * N + N + t] = b;
  }
  __syncthreads();
}

// Stage T^T/(N-1) scaled per column (ts_j = 1/rms_k(T_kj/(N-1))) into the B operand of the
// u MMA (rows j, K-major over k); also the FP64 column norms ||T_:j||^2.
template <typename T16, int NT, int TERMS>
__device__ __forceinline__ void stage_Tt16(const double* __restrict__ Tred, int N, double inv,
                                           T16* sBu, float* ts, double* tn2, double* scratch) {
  constexpr int L = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, k0 = t / NT;
  double nrm = 0.0;
  for (int k = k0; k < NT; k += L) {
    const double v = (k < N && j < N) ? __ldcg(Tred + k * N + j) : 0.0;
    nrm = fma(v, v, nrm);
  }
  scratch[t] = nrm;
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < L; ++q) s += scratch[q * NT + t];
    tn2[t] = s;
    const double rms = sqrt(s / (double)(N > 0 ? N : 1)) * inv;
    ts[t] = (t < N && rms > 0.0) ? (float)(1.0 / rms) : 1.f;
  }
  __syncthreads();
  for (int e = t; e < NT * NT; e += kThreads) {
    const int jj = e / NT, k = e % NT;
    const double v = (k < N && jj < N) ? __ldcg(Tred + k * N + jj) * inv * (double)ts[jj] : 0.0;
    const T16 hi = H16<T16>::from((float)v);
    sBu[core_idx(jj, k, NT)] = hi;
    if (TERMS == 3) sBu[NT * NT + core_idx(jj, k, NT)] = H16<T16>::from((float)(v - (double)(float)hi));
  }
  fence_async_smem();
  __syncthreads();
}

struct MixedParams {
  int64_t m;
  int N;
  const void* HA16;
  const float* HA32;
  const df32* HAdf;
  const df32* Ddf;
  df32* Zdf;
  const double* D;
  float* B;         // right-hand side of the current inner solve (D, then refreshed residuals)
  const double* r;
  const float* r32;
  float* X;
  float* Res;
  float* P;
  float* Sv;
  double* Tpart;
  double* Tred;
  double* rrpart;
  double* W;
  double tol, inner_tol, itol_floor;
  int max_iter, refresh_every;
  int* col_iters;
  double* col_relres;
  double* col_true;
  int* status;
  unsigned* bar;
};

template <typename T16, int NT, bool PC, int TERMS>
__global__ void __launch_bounds__(kThreads, 1) solve_mixed_kernel(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  double* s_gam = reinterpret_cast<double*>(smem);
  double* s_gold = s_gam + NT;
  double* s_sig = s_gold + NT;
  double* s_tn2 = s_sig + NT;
  double* s_bn2 = s_tn2 + NT;
  double* s_dn2 = s_bn2 + NT;
  double* s_alpha = s_dn2 + NT;
  double* s_beta = s_alpha + NT;
  double* s_prev = s_beta + NT;
  double* s_tmp = s_prev + NT;
  double* s_true = s_tmp + NT;
  double* s_rel = s_true + NT;
  int* s_active = reinterpret_cast<int*>(s_rel + NT);
  int* s_done = s_active + NT;
  int* s_iters = s_done + NT;
  int* s_flag = s_iters + NT;
  float* s_alpha_v = reinterpret_cast<float*>(s_flag + NT);
  float* s_beta_v = s_alpha_v + NT;
  float* s_itol = s_beta_v + NT;   // per-column inner-solve reduction factor
  double* scratch = reinterpret_cast<double*>(smem + scalar_bytes<NT>());
  unsigned char* uni = smem + scalar_bytes<NT>() + kThreads * 8;
  // tensor-core operands (inside the union; the FP32 refresh passes reuse the same bytes)
  constexpr int TM = TERMS == 3 ? 2 : 1;   // hi (+ lo) copies of every operand tile
  T16* sAu = reinterpret_cast<T16*>(uni);
  T16* sBu = sAu + TM * kTR * NT;
  T16* sAg = sBu + TM * NT * NT;
  T16* sBg = sAu;   // the z operand of the Gram MMA is written after the u MMA has read sAu
  float* sacc = reinterpret_cast<float*>(sAg + TM * kTR * kTR);
  float* s_zs = sacc + 8 * 2 * NT;
  float* s_ts = s_zs + NT;

  const int N = p.N, G = gridDim.x, b = blockIdx.x, t = threadIdx.x, warp = t >> 5;
  const int64_t rows_per = (p.m + G - 1) / G;
  const int64_t row0 = imin64(p.m, (int64_t)b * rows_per);
  const int64_t row1 = imin64(p.m, row0 + rows_per);
  const int NE = N * N + 2 * N;
  GridBarrier bar{p.bar, reinterpret_cast<int*>(p.bar + 1), p.status, (unsigned)G, 0u};
  const double inv_nm1 = 1.0 / (double)(N - 1);
  double* Tp = p.Tpart + (int64_t)b * NE;
  const T16* HAhi = static_cast<const T16*>(p.HA16);
  const T16* HAlo = HAhi + p.m * (int64_t)N;
  constexpr int TMC = tc_tmem_cols<NT>();

  if (t == 0) { mbar_init(&mbar[0]); mbar_init(&mbar[1]); }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)), "r"(TMC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t ph_u = 0, ph_g = 0;
  int par = 0;
  bool ok = true;

  // ---- ||d_j||^2 (FP64) and Z = 0 (double-float solution accumulator)
  rows_reduce<NT>(row0, row1, N, [&](int64_t i, int j, double& acc) {
    const double d = p.D[i * N + j];
    acc = fma(d, d, acc);
    p.Zdf[i * N + j] = df32(0.f, 0.f);
  }, s_tmp, scratch);
  if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
  ok = bar.sync();
  if (ok) {
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_dn2, scratch);
    par ^= 1;
    if (t < NT) {
      s_done[t] = (t >= N || s_dn2[t] == 0.0) ? 1 : 0;
      s_iters[t] = 0;
      s_true[t] = (t < N && s_dn2[t] == 0.0) ? 0.0 : -1.0;
      s_rel[t] = (t < N && s_dn2[t] > 0.0) ? 1.0 : 0.0;
      s_prev[t] = 2.0;
      s_alpha_v[t] = 0.f;
      s_beta_v[t] = 0.f;
      s_itol[t] = (float)fmax(p.inner_tol, p.itol_floor);
    }
    __syncthreads();
  }
  int total = 0, cycles = 0;
  while (ok) {
    // ---- inner solve of S X = B from X = 0: first reduction of [HA^T z | slot A | slot B]
    {
      ProSetup<float, PC> pro{p.B, p.X, p.Res, p.r32, N};
      passA<float, NT, ProSetup<float, PC>, PC>(p.HA32, row0, row1, N, p.r32, true, pro, uni, Tp);
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b);
    if (!(ok = bar.sync())) break;
    stage_Tt16<T16, NT, TERMS>(p.Tred, N, inv_nm1, sBu, s_ts, s_tn2, scratch);
    if (t < NT) {
      const double sg = t < N ? __ldcg(p.Tred + N * N + t) : 0.0;
      const double gm = t < N ? __ldcg(p.Tred + N * N + N + t) : 0.0;
      s_sig[t] = sg;
      s_gam[t] = gm;
      s_bn2[t] = gm;   // residual norm^2 at the start of this inner solve
      s_active[t] = (t < N && !s_done[t] && gm > 0.0) ? 1 : 0;
      s_alpha[t] = 0.0;
      s_beta[t] = 0.0;
    }
    __syncthreads();
    int it = 0;
    for (;;) {
      if (t < NT) {
        int a = s_active[t];
        const double gm = s_gam[t];
        double al = 0.0, be = 0.0;
        if (a && !isfinite(gm)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
        // the inner solve of this column ends once its residual fell by the factor s_itol
        if (a && it > 0 && sqrt(gm) <= s_itol[t] * sqrt(s_bn2[t])) a = 0;
        if (a) {
          const double cg = PC ? s_sig[t] : gm;
          const double delta = s_tn2[t] * inv_nm1 + s_sig[t];
          double den = delta;
          if (it > 0) {
            be = cg / s_gold[t];
            den = delta - be * cg / s_alpha[t];
          }
          // p^T S p = delta - beta gamma/alpha_old cancels; with BF16/FP16 contractions a
          // small or non-positive value means the low-precision recurrences have drifted:
          // this column's inner solve ends here and the refresh restarts it
          if (!isfinite(den) || !(den > 0.05 * delta)) { a = 0; be = 0.0; }
          else al = cg / den;
        }
        s_active[t] = a;
        s_alpha[t] = al;
        s_beta[t] = be;
        s_alpha_v[t] = (float)al;
        s_beta_v[t] = (float)be;
        s_zs[t] = (t < N && gm > 0.0) ? (float)(1.0 / sqrt(gm)) : 1.f;
      }
      __syncthreads();
      if (t == 0) {
        int any = 0;
        for (int j = 0; j < N; ++j) any |= s_active[j];
        s_flag[0] = any && (p.refresh_every <= 0 || it < p.refresh_every) && total + it < p.max_iter;
      }
      __syncthreads();
      if (!s_flag[0]) break;
      passF_tc<T16, NT, PC, TERMS>(HAhi, HAlo, row0, row1, N, p.X, p.Res, p.P, p.Sv, p.r32, s_alpha_v,
                                   s_beta_v, s_zs, s_ts, sAu, sBu, sAg, sBg, sacc, tmem, &mbar[0],
                                   &mbar[1], ph_u, ph_g, p.status, ok, Tp);
      if (!(ok = bar.sync() && ok)) break;
      reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b);
      if (!(ok = bar.sync())) break;
      stage_Tt16<T16, NT, TERMS>(p.Tred, N, inv_nm1, sBu, s_ts, s_tn2, scratch);
      if (t < N && s_active[t]) {
        s_iters[t] += 1;
        s_gold[t] = PC ? s_sig[t] : s_gam[t];
        s_gam[t] = __ldcg(p.Tred + N * N + N + t);
        s_sig[t] = __ldcg(p.Tred + N * N + t);
      }
      __syncthreads();
      ++it;
    }
    if (!ok) break;
    total += it;
    ++cycles;
    // ---- double-float refresh: Z += X; T = HA^T Z; W; true residual D - S Z -> next B
    {
      ProRefreshDF<float> pro{p.Zdf, p.X, N, true};
      passA<df32, NT>(p.HAdf, row0, row1, N, static_cast<const df32*>(nullptr), false, pro, uni, Tp);
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b);
    if (!(ok = bar.sync())) break;
    if (b == 0)
      for (int e = t; e < N * N; e += kThreads) p.W[e] = __ldcg(p.Tred + e) * inv_nm1;
    {
      df32* sTd = reinterpret_cast<df32*>(uni);
      stage_T<df32, NT>(p.Tred, N, sTd);
      constexpr int LDD = NT + 2;
      EpiRefreshDF<float> epi{p.Zdf, p.Ddf, p.r, p.B, N, df32(inv_nm1)};
      passB<df32, NT>(p.HAdf, row0, row1, N, sTd, uni + NT * LDD * sizeof(df32), epi, s_tmp);
    }
    if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
    if (!(ok = bar.sync())) break;
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_tmp, scratch);
    par ^= 1;
    if (t < N) {
      const double rel = s_dn2[t] > 0.0 ? sqrt(s_tmp[t] / s_dn2[t]) : 0.0;
      s_rel[t] = rel;
      s_true[t] = rel;
      if (!s_done[t]) {
        // converged, or stalled (no halving over a cycle)
        if (rel <= p.tol || (cycles >= 2 && rel > 0.5 * s_prev[t])) s_done[t] = 1;
      }
      s_prev[t] = rel;
      // the next inner solve only has to gain the remaining factor tol/rel (margin 0.1),
      // but not more than the low-precision operator allows
      double it_next = rel > 0.0 ? 0.1 * p.tol / rel : 0.5;
      it_next = fmax(it_next, fmax(p.inner_tol, p.itol_floor));
      s_itol[t] = (float)fmin(it_next, 0.5);
    }
    __syncthreads();
    if (t == 0) {
      int all = 1;
      for (int j = 0; j < N; ++j) all &= s_done[j];
      s_flag[1] = all || total >= p.max_iter;
    }
    __syncthreads();
    if (s_flag[1]) break;
  }

  if (b == 0 && t < N) {
    p.col_iters[t] = s_iters[t];
    p.col_relres[t] = s_rel[t];
    p.col_true[t] = s_true[t];
    if (ok && !(s_rel[t] <= p.tol)) atomicOr(p.status, DS_NOT_CONVERGED);
  }
  if (b == 0 && t == 0) p.status[1] = cycles;
  // release tensor memory on every path
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMC));
}

template <int NT, int TERMS> __host__ __device__ constexpr int mixed_smem_bytes() {
  constexpr int u = refresh_union_bytes<NT>() > tc_bytes<NT, TERMS>() ? refresh_union_bytes<NT>() : tc_bytes<NT, TERMS>();
  return scalar_bytes<NT>() + kThreads * 8 + u;
}

}  // namespace enkf
