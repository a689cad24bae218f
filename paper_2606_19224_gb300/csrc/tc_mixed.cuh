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
// Operands sit in shared memory in the canonical no-swizzle core-matrix layout (8 rows x 16
// bytes per core matrix). For a K-major operand the descriptor's LBO is the K-direction core
// stride and SBO the row-group stride; for an MN-major one (16-bit elements contiguous along
// M or N) LBO is again the K-direction core stride and SBO the MN-direction one. One thread
// issues the MMAs; completion is signalled through an mbarrier by tcgen05.commit; every wait
// is bounded.
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
// kind::f16 instruction descriptor: D F32, A = B = F16 (fmt 0) or BF16 (fmt 1), A K-major,
// B K-major (b_mn = false) or MN-major (bit 16), dense, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc(uint32_t fmt, int N, bool b_mn = false) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
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
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t phase, int* status,
                                          unsigned long long timeout_ns = kBarrierTimeoutNs) {
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  while (!done) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_addr(mbar)), "r"(phase));
    if (!done && global_ns() - t0 > timeout_ns) {
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
  __device__ static float to(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <> struct H16<__half> {
  static constexpr uint32_t fmt = 0;
  __device__ static __half from(float x) { return __float2half_rn(x); }
  __device__ static float to(__half x) { return __half2float(x); }
};

// element (r, k) of a K-major operand with Kd K-elements per row, in elements of 2 bytes:
// core matrix (r/8, k/8) at ((r/8)*(Kd/8) + k/8) * 64, then (r%8)*8 + k%8
__device__ __forceinline__ int core_idx(int r, int k, int Kd) {
  return (((r >> 3) * (Kd >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

constexpr int kTR = 128;  // rows per tile = M of the u MMA = K of the Gram MMA

// two 16-bit values as one 32-bit word, `a` at the lower address
template <typename T16> __device__ __forceinline__ uint32_t pack16(T16 a, T16 b) {
  return (uint32_t)reinterpret_cast<const uint16_t&>(a) | ((uint32_t)reinterpret_cast<const uint16_t&>(b) << 16);
}

// TMEM columns (a power of two >= 32): NT <= 64 keeps two u slots and the Gram (3 NT), NT = 128
// one u and the Gram (2 NT)
template <int NT> __host__ __device__ constexpr int tc_tmem_cols() { return NT <= 32 ? 128 : (NT <= 64 ? 256 : 2 * NT); }

// ------------------------------------------------------------------ fused tensor-core CG step
// Same recurrences as passF (Chronopoulos-Gear arrangement, optionally preconditioned by R);
// the contractions run on the tensor cores. Bu holds (T/(N-1)) scaled per column by ts_j and
// the z operand holds z scaled per column by zs_j (so FP16 neither overflows nor flushes);
// the scales are undone on the FP32 values read from TMEM.
// TERMS == 3: every operand is split into x_hi = round(x) and x_lo = round(x - x_hi) and each
// product is formed as hi*hi + hi*lo + lo*hi (three MMAs into the same accumulator), about 16
// significant bits instead of 8 (BF16) or 11 (FP16).
//
// HA reaches the CTA as precomputed tile images (tc_images_kernel): for every 128-row tile of
// the CTA's row block, [hi | lo] in the K-major core layout of the tile's rows (128 x NT), so
// staging a tile is a plain 16-byte cp.async copy. The same image serves both MMAs: as the
// K-major A operand of u = HA T (M = 128 rows, K = NT) and as the MN-major B operand of the
// Gram D_g[j][k] = sum_i z_ij HA_ik (N = NT along k, K = the tile's 128 rows), whose A operand
// is z^T scaled per column (M = 128, rows j >= N zero). One image instead of one per MMA keeps
// the working set (images and CG vectors) in L2.
// NT <= 64: two image buffers (the next tile's copy overlaps the whole current tile), the u
// read-out staged as FP32 in its own region, the z operand with a padded K-direction core
// stride (144 B, conflict-free stores), and the column sums of (r, z) and (r, r) in registers
// until the end of the pass. NT = 128: one image buffer, refilled once the Gram MMA is done.
template <int NT, int TERMS> struct TcLayout {
  static constexpr int TM = TERMS == 3 ? 2 : 1;
  static constexpr bool DB = NT <= 64;
  static constexpr int AU = kTR * NT, BU = NT * NT;                  // elements per part
  static constexpr int TILE = TM * AU;                               // elements per tile image
  static constexpr int AUB = TILE * 2;                               // bytes per tile image
  // z operand strides. NT <= 64: each warp writes one row i across 64 columns j, so the
  // j-direction core stride is 16 B off a multiple of 128 B (2-way bank conflicts at most,
  // against 8-way with a 128-B multiple); NT = 128: each warp writes 32 rows i of one column,
  // K-direction core stride 128 B (smem is too tight for padding there).
  static constexpr uint32_t LBOG = 128;                              // z operand: K core stride
  static constexpr uint32_t SBOG = DB ? 16 * LBOG + 16 : 16 * LBOG;  // M core stride
  static constexpr int BGP = (int)(16 * SBOG);                       // bytes per z part (M = 128)
  static constexpr int n_au = DB ? 2 : 1;
  static constexpr int off_au = 0;
  static constexpr int off_bu = off_au + n_au * AUB;
  static constexpr int off_bg = off_bu + TM * BU * 2;
  static constexpr int end_bg = off_bg + TM * BGP;
  static constexpr int off_sacc = end_bg;
  static constexpr int off_zs = off_sacc + 4 * (8 * 2 * NT);
  static constexpr int off_ts = off_zs + 4 * NT;   // ts [NT] then 1/ts [NT]
  // NT <= 64: the tile's u = HA T read out of TMEM, staged as FP32 [128][NT] (swizzled 4-float
  // groups) for the coalesced epilogue
  static constexpr int off_u = off_ts + 8 * NT;
  // NT <= 64: T_k of the Hestenes-Stiefel recurrence, FP32 [NT][NT] (stage_Tt16_rec)
  static constexpr int off_tk = off_u + kTR * NT * 4;
  // NT <= 64: the pass's Gram summed over its tiles in FP32, [NT][NT + 1] (row j, column k)
  static constexpr int off_gacc = off_tk + NT * NT * 4;
  static constexpr int bytes = DB ? off_gacc + NT * (NT + 1) * 4 : off_ts + 8 * NT;
  static_assert(off_bu % 1024 == 0 && off_bg % 1024 == 0 && off_u % 16 == 0, "operand alignment");
};

__device__ __forceinline__ void tc_cp16(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void tc_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void tc_cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// copy `bytes` (a multiple of 16) from global to shared with all threads of the CTA
__device__ __forceinline__ void tc_copy(unsigned char* sdst, const unsigned char* gsrc, int bytes) {
  for (int o = threadIdx.x * 16; o < bytes; o += kThreads * 16) tc_cp16(sdst + o, gsrc + o);
}

template <typename T16, int NT, bool PC, int TERMS>
__device__ void passF_tc2(const T16* __restrict__ img, int qmax, int64_t row0, int64_t row1, int N,
                          float* X, float* Res, float* P, const float* __restrict__ rv,
                          const float* alpha, const float* beta, unsigned char* tcs, uint32_t tmem,
                          uint64_t* mbar_u, uint64_t* mbar_g, uint32_t& ph_u, uint32_t& ph_g, int* status,
                          bool& ok, double* __restrict__ out, float gsi) {
  using L = TcLayout<NT, TERMS>;
  constexpr bool SPLIT = TERMS == 3, DB = L::DB;
  static_assert(!DB, "NT = 128 only");
  constexpr uint32_t idesc = umma_idesc(H16<T16>::fmt, NT);
  constexpr uint32_t idesc_g = umma_idesc(H16<T16>::fmt, NT, true);
  constexpr int HALF = NT / 2, CH = HALF / 16;   // columns per warp half, 16-column chunks
  T16* sAu = reinterpret_cast<T16*>(tcs + L::off_au);
  const T16* sBu = reinterpret_cast<const T16*>(tcs + L::off_bu);
  unsigned char* sBg = tcs + L::off_bg;
  float* sacc = reinterpret_cast<float*>(tcs + L::off_sacc);
  const float* zs = reinterpret_cast<const float*>(tcs + L::off_zs);
  const float* ts = reinterpret_cast<const float*>(tcs + L::off_ts);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int qd = warp & 3, half = warp >> 2;
  const int rt = 32 * qd + lane;                 // the thread's row within the tile (TMEM lane)
  const bool vec = (N & 3) == 0;
  const uint32_t d_u = tmem, d_g = tmem + NT;
  const int Qb = row1 > row0 ? (int)((row1 - row0 + kTR - 1) / kTR) : 0;
  const unsigned char* gimg = reinterpret_cast<const unsigned char*>(img);
  auto au_src = [&](int q) { return gimg + (size_t)q * L::AUB; };
  // z operand element (row j, col i) of part `part`
  auto bg_ptr = [&](int part, int j, int i) {
    return reinterpret_cast<T16*>(sBg + part * L::BGP + (j >> 3) * L::SBOG + (i >> 3) * L::LBOG +
                                  (((j & 7) * 8 + (i & 7)) * 2));
  };
  (void)qmax;
  // column sums [(r, z) | (r, r) | sum r_i z^2 | sum r_i z p] of the pass, one slot per warp
  // quarter (a column is handled by the four warps of one half): sacc[(c * 4 + qd) * NT + j]
  for (int e = t; e < 4 * 4 * NT; e += kThreads) sacc[e] = 0.f;
  if (Qb > 0) {
    tc_copy(reinterpret_cast<unsigned char*>(sAu), au_src(0), L::AUB);
    tc_cp_commit();
  }
  for (int q = 0; q < Qb && ok; ++q) {
    const int64_t i0 = row0 + (int64_t)q * kTR;
    tc_cp_wait_all();
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      constexpr uint32_t sbo_u = (NT / 8) * 128;
      const uint32_t au = smem_addr(sAu), bu = smem_addr(sBu);
      // split operands: the small cross terms hi*lo + lo*hi first, then hi*hi, so that each
      // addition into the FP32 accumulator rounds against the smaller partial sum first
      if (SPLIT) {
#pragma unroll
        for (int kb = 0; kb < NT / 16; ++kb) {
          umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + 2 * L::BU + kb * 256, 128, sbo_u), idesc, kb > 0 ? 1u : 0u);
          umma_f16(d_u, umma_desc(au + 2 * L::AU + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc, 1u);
        }
      }
#pragma unroll
      for (int kb = 0; kb < NT / 16; ++kb)
        umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc,
                 (kb > 0 || SPLIT) ? 1u : 0u);
      umma_commit(mbar_u);
    }
    const int64_t i = i0 + rt;
    const bool valid = i < row1;
    const float ri = valid ? rv[i] : 1.f;
    const float rinv = 1.f / ri;
    // operands of the first chunk are loaded while the MMA runs
    float rr[16], pp[16], xx[16];
    auto load_chunk = [&](int j0) {
#pragma unroll
      for (int y4 = 0; y4 < 4; ++y4) {
        const int jj = j0 + 4 * y4;
        float a[4] = {0.f, 0.f, 0.f, 0.f}, bq[4] = {0.f, 0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f};
        if (valid && jj < N) {
          ld4<float>(a, Res + i * N, jj, N, vec);
          ld4<float>(bq, P + i * N, jj, N, vec);
          ld4<float>(dq, X + i * N, jj, N, vec);
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          rr[4 * y4 + y] = a[y];
          pp[4 * y4 + y] = bq[y];
          xx[4 * y4 + y] = dq[y];
        }
      }
    };
    load_chunk(half * HALF);
    if (!mbar_wait(mbar_u, ph_u, status)) ok = false;
    ph_u ^= 1u;
    tc_fence_after();
    float tS[4][16];   // this chunk's column terms, reduced over the warp per chunk
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j0 = half * HALF + 16 * c;
      if (c > 0) load_chunk(j0);
      float u[16];
      tmem_ld16(d_u + ((uint32_t)(32 * qd) << 16) + j0, u);
      float pn[16], xn[16], rn[16];
#pragma unroll
      for (int y = 0; y < 16; ++y) {
        const int j = j0 + y;
        // the step of passH: p = z + beta p, q = HA T/(N-1) + r_i p, x += alpha p, r -= alpha q
        const float uu = u[y] * ts[NT + j];
        const float zz = PC ? rr[y] * rinv : rr[y];
        const float be = beta[j], al = alpha[j];
        pn[y] = be == 0.f ? zz : fmaf(be, pp[y], zz);
        const float qq = fmaf(ri, pn[y], uu);
        xn[y] = fmaf(al, pn[y], xx[y]);
        rn[y] = fmaf(-al, qq, rr[y]);
        const float zn = PC ? rn[y] * rinv : rn[y];
        const bool live = valid && j < N;
        tS[0][y] = live ? rn[y] * zn : 0.f;
        tS[1][y] = live ? rn[y] * rn[y] : 0.f;
        tS[2][y] = live ? ri * zn * zn : 0.f;
        tS[3][y] = live ? ri * zn * pn[y] : 0.f;
        const float zsc = live ? zn * zs[j] : 0.f;
        const T16 zh = H16<T16>::from(zsc);
        *bg_ptr(0, j, rt) = zh;
        if (SPLIT) *bg_ptr(1, j, rt) = H16<T16>::from(zsc - (float)zh);
      }
      if (valid) {
#pragma unroll
        for (int y4 = 0; y4 < 4; ++y4) {
          const int jj = j0 + 4 * y4;
          if (jj < N) {
            const float o1[4] = {pn[4 * y4], pn[4 * y4 + 1], pn[4 * y4 + 2], pn[4 * y4 + 3]};
            const float o3[4] = {xn[4 * y4], xn[4 * y4 + 1], xn[4 * y4 + 2], xn[4 * y4 + 3]};
            const float o4[4] = {rn[4 * y4], rn[4 * y4 + 1], rn[4 * y4 + 2], rn[4 * y4 + 3]};
            st4<float>(P + i * N, jj, N, vec, o1);
            st4<float>(X + i * N, jj, N, vec, o3);
            st4<float>(Res + i * N, jj, N, vec, o4);
          }
        }
      }
      // this chunk's per-column sums over the warp's 32 rows, into the warp quarter's slot
#pragma unroll
      for (int cc = 0; cc < 4; ++cc)
#pragma unroll
        for (int y = 0; y < 16; ++y) {
          float a = tS[cc][y];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
          if (lane == 0) sacc[(cc * 4 + qd) * NT + j0 + y] += a;
        }
    }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      // B = the tile image read MN-major: K = rows (row-group stride (NT/8) 128 B, two per
      // K block of 16), N = NT (core stride 128 B)
      const uint32_t au = smem_addr(sAu), bg = smem_addr(sBg);
      constexpr uint32_t kst = (NT / 8) * 128;
      // split operands: the cross terms of the tile first, then hi*hi
      if (SPLIT) {
#pragma unroll
        for (int kb = 0; kb < kTR / 16; ++kb) {
          const uint64_t A0 = umma_desc(bg + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
          const uint64_t B0 = umma_desc(au + kb * 2 * kst, kst, 128);
          const uint64_t A1 = umma_desc(bg + L::BGP + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
          const uint64_t B1 = umma_desc(au + L::AU * 2 + kb * 2 * kst, kst, 128);
          umma_f16(d_g, A0, B1, idesc_g, (q == 0 && kb == 0) ? 0u : 1u);
          umma_f16(d_g, A1, B0, idesc_g, 1u);
        }
      }
#pragma unroll
      for (int kb = 0; kb < kTR / 16; ++kb) {
        const uint64_t A0 = umma_desc(bg + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
        const uint64_t B0 = umma_desc(au + kb * 2 * kst, kst, 128);
        umma_f16(d_g, A0, B0, idesc_g, (q == 0 && kb == 0 && !SPLIT) ? 0u : 1u);
      }
      umma_commit(mbar_g);
    }
    // the Gram MMA reads the z operand and the image: wait before either is rewritten
    if (!mbar_wait(mbar_g, ph_g, status)) ok = false;
    ph_g ^= 1u;
    tc_fence_after();
    if (q + 1 < Qb) {
      tc_copy(reinterpret_cast<unsigned char*>(sAu), au_src(q + 1), L::AUB);
      tc_cp_commit();
    }
  }
  tc_cp_wait_all();
  // partial Gram from TMEM: D_g lane j, column k -> out[k*N + j] / zs_j (the condition is
  // uniform within a warp: tcgen05.ld is warp-collective)
  if (Qb > 0 && 32 * qd < N) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int k0 = half * HALF + 16 * c;
      float v[16];
      tmem_ld16(d_g + ((uint32_t)(32 * qd) << 16) + k0, v);
      if (rt < N) {
        const float inv = gsi / zs[rt];
#pragma unroll
        for (int y = 0; y < 16; ++y)
          if (k0 + y < N) out[(k0 + y) * N + rt] = (double)(v[y] * inv);
      }
    }
  } else if (Qb == 0) {
    for (int e = t; e < N * N; e += kThreads) out[e] = 0.0;
  }
  tc_fence_before();
  __syncthreads();
  if (t < N) {
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double a = 0.0;
      for (int w = 0; w < 4; ++w) a += (double)sacc[(cc * 4 + w) * NT + t];
      out[N * N + cc * N + t] = a;
    }
  }
  __syncthreads();
}

// NT <= 64: the same step with a coalesced epilogue. The tile's u = HA T leaves TMEM row by
// row (thread = row) into an FP32 staging tile (4-float groups XOR-swizzled by row, so both
// the row-wise writes and the group-wise reads are free of bank conflicts); the CG update
// then runs with NT/4 threads per row on 16-byte column groups, so the loads and stores of
// r, p, S p and x are contiguous 256-byte row segments, and each thread keeps the (r, z) and
// (r, r) sums of its four columns in registers for the whole pass.
template <typename T16, int NT, bool PC, int TERMS>
__device__ void passF_tc_db(const T16* __restrict__ img, int64_t row0, int64_t row1, int N, float* X,
                            float* Res, float* P, const float* __restrict__ rv,
                            const float* alpha, const float* beta, unsigned char* tcs, uint32_t tmem,
                            uint64_t* mbar_u2, uint64_t* mbar_g, uint32_t* ph_u2, uint32_t& ph_g,
                            int* status, bool& ok, double* __restrict__ out, bool atomic_out, float gsi) {
  using L = TcLayout<NT, TERMS>;
  static_assert(L::DB, "NT <= 64 only");
  constexpr bool SPLIT = TERMS == 3;
  constexpr int TM = L::TM;
  constexpr uint32_t idesc = umma_idesc(H16<T16>::fmt, NT);
  constexpr uint32_t idesc_g = umma_idesc(H16<T16>::fmt, NT, true);
  constexpr int HALF = NT / 2, CH = HALF / 16;    // TMEM read-out: columns per warp half
  constexpr int NG = NT / 4, GM = NG - 1;         // 4-float column groups, swizzle mask
  constexpr int NJ = NG, RI = kThreads / NJ;      // update: threads per row, rows per sweep
  constexpr int SWEEPS = kTR / RI, SMID = SWEEPS / 2;
  constexpr uint32_t sbo_u = (NT / 8) * 128;
  unsigned char* sAu0 = tcs + L::off_au;
  const T16* sBu = reinterpret_cast<const T16*>(tcs + L::off_bu);
  unsigned char* sBg = tcs + L::off_bg;
  float* sU = reinterpret_cast<float*>(tcs + L::off_u);
  const float* zs = reinterpret_cast<const float*>(tcs + L::off_zs);
  const float* ts = reinterpret_cast<const float*>(tcs + L::off_ts);
  float* sG = reinterpret_cast<float*>(tcs + L::off_gacc);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int qd = warp & 3, half = warp >> 2;
  const int rt = 32 * qd + lane;
  const int tj = t % NJ, ti = t / NJ, j0 = 4 * tj;
  // The Gram of each tile leaves TMEM once it is complete and is added to sG in FP32 (round to
  // nearest), so no tensor-core accumulation chain spans more than one tile: a chain over all
  // of a CTA's tiles cost the split FP16 mode steps and a refresh (more with fewer, longer
  // row blocks). Thread (qd, half, lane) owns row j = 32 qd + lane, columns [half NT/2, +NT/2).
  const bool g_owner = 32 * qd < N;
  auto gram_out = [&]() {
    if (!g_owner) return;
#pragma unroll
    for (int c = 0; c < HALF / 16; ++c) {
      const int k0 = half * HALF + 16 * c;
      float v[16];
      tmem_ld16(tmem + 2 * NT + ((uint32_t)(32 * qd) << 16) + k0, v);
#pragma unroll
      for (int y = 0; y < 16; ++y) sG[rt * (NT + 1) + k0 + y] += v[y];
    }
  };
  if (g_owner)
    for (int k = half * HALF; k < half * HALF + HALF; ++k) sG[rt * (NT + 1) + k] = 0.f;
  // TMEM: u of tile q in slot q % 2 (columns [slot NT, slot NT + NT)), the Gram at 2 NT
  const uint32_t d_g = tmem + 2 * NT;
  const int Qb = row1 > row0 ? (int)((row1 - row0 + kTR - 1) / kTR) : 0;
  const unsigned char* gimg = reinterpret_cast<const unsigned char*>(img);
  auto au_src = [&](int q) { return gimg + (size_t)q * L::AUB; };
  auto sAu = [&](int q) { return sAu0 + (q & 1) * L::AUB; };
  auto bg_ptr = [&](int part, int j, int i) {
    return reinterpret_cast<T16*>(sBg + part * L::BGP + (j >> 3) * L::SBOG + (i >> 3) * L::LBOG +
                                  (((j & 7) * 8 + (i & 7)) * 2));
  };
  // u = HA T of tile q (image in buffer q % 2) into TMEM slot q % 2, completion on mbar_u2[q % 2]
  auto issue_u = [&](int q) {
    tc_fence_after();
    const uint32_t au = smem_addr(sAu(q)), bu = smem_addr(sBu);
    const uint32_t d_u = tmem + (uint32_t)((q & 1) * NT);
    // split operands: the small cross terms first, then hi*hi (as in passF_tc2)
    if (SPLIT) {
#pragma unroll
      for (int kb = 0; kb < NT / 16; ++kb) {
        umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + 2 * L::BU + kb * 256, 128, sbo_u), idesc, kb > 0 ? 1u : 0u);
        umma_f16(d_u, umma_desc(au + 2 * L::AU + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc, 1u);
      }
    }
#pragma unroll
    for (int kb = 0; kb < NT / 16; ++kb)
      umma_f16(d_u, umma_desc(au + kb * 256, 128, sbo_u), umma_desc(bu + kb * 256, 128, sbo_u), idesc,
               (kb > 0 || SPLIT) ? 1u : 0u);
    umma_commit(&mbar_u2[q & 1]);
  };
  // per-column constants of the thread's four columns
  float al[4], be[4], tsi[4], zsc[4];
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    al[y] = alpha[j0 + y];
    be[y] = beta[j0 + y];
    tsi[y] = ts[NT + j0 + y];
    zsc[y] = zs[j0 + y];
  }
  // rows j in [NT, 128) of the z operand stay zero for the whole pass
  for (int e = t; e < TM * (kTR - NT) * kTR; e += kThreads) {
    const int part = e / ((kTR - NT) * kTR), rem = e % ((kTR - NT) * kTR);
    *bg_ptr(part, NT + rem / kTR, rem % kTR) = H16<T16>::from(0.f);
  }
  float s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
  float s3[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f};
  const bool vec = (N & 3) == 0;
  // the operands of one row sweep of the update: r, p, x of the thread's four columns and r_i
  struct Ops { float rr[4], pp[4], xx[4], ri; };
  auto load_ops = [&](int64_t i0, int r, Ops& o) {
    const int64_t i = i0 + r;
#pragma unroll
    for (int y = 0; y < 4; ++y) { o.rr[y] = 0.f; o.pp[y] = 0.f; o.xx[y] = 0.f; }
    o.ri = 1.f;
    if (i < row1 && j0 < N) {
      ld4<float>(o.rr, Res + i * N, j0, N, vec);
      ld4<float>(o.pp, P + i * N, j0, N, vec);
      ld4<float>(o.xx, X + i * N, j0, N, vec);
      o.ri = rv[i];
    }
  };
  // Pipeline over the CTA's tiles: u of tile q + 1 is issued half-way through the update of
  // tile q (its image is copied at the start of tile q, once the Gram of tile q - 1, the last
  // reader of that buffer, has completed); the Gram of tile q runs behind the read-out of
  // tile q + 1 and is waited for only before the z operand is rewritten.
  if (Qb > 0) {
    tc_copy(sAu(0), au_src(0), L::AUB);
    tc_cp_commit();
    tc_cp_wait_all();
    fence_async_smem();
    __syncthreads();
    if (t == 0) issue_u(0);
  }
  for (int q = 0; q < Qb && ok; ++q) {
    const int64_t i0 = row0 + (int64_t)q * kTR;
    // every sweep's operands of this tile, in flight during the wait and the read-out (one
    // L2 round trip per tile instead of one per sweep)
    Ops ops[SWEEPS];
#pragma unroll
    for (int sw = 0; sw < SWEEPS; ++sw) load_ops(i0, ti + sw * RI, ops[sw]);
    if (!mbar_wait(&mbar_u2[q & 1], ph_u2[q & 1], status)) ok = false;
    ph_u2[q & 1] ^= 1u;
    tc_fence_after();
    // u out of TMEM, one row per thread, into the swizzled staging tile
    const uint32_t d_u = tmem + (uint32_t)((q & 1) * NT);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int jc = half * HALF + 16 * c;
      float v[16];
      tmem_ld16(d_u + ((uint32_t)(32 * qd) << 16) + jc, v);
#pragma unroll
      for (int g4 = 0; g4 < 4; ++g4) {
        const int pg = ((jc >> 2) + g4) ^ (rt & GM);
        *reinterpret_cast<float4*>(sU + rt * NT + pg * 4) =
            make_float4(v[4 * g4], v[4 * g4 + 1], v[4 * g4 + 2], v[4 * g4 + 3]);
      }
    }
    tc_fence_before();
    __syncthreads();
    // the Gram of tile q - 1 reads the z operand and the image buffer of tile q + 1
    if (q > 0) {
      if (!mbar_wait(mbar_g, ph_g, status)) ok = false;
      ph_g ^= 1u;
      tc_fence_after();
      gram_out();
    }
    const bool more = q + 1 < Qb;
    if (more) {
      tc_copy(sAu(q + 1), au_src(q + 1), L::AUB);
      tc_cp_commit();
    }
    // the CG update, NT/4 threads per row
#pragma unroll
    for (int sw = 0; sw < SWEEPS; ++sw) {
      const int r = ti + sw * RI;
      if (sw == SMID && more) {
        // the next tile's image has had half a tile to land: start its u MMA
        tc_cp_wait_all();
        fence_async_smem();
        __syncthreads();
        if (t == 0) issue_u(q + 1);
      }
      const int64_t i = i0 + r;
      const bool valid = i < row1 && j0 < N;
      const Ops& cur = ops[sw];
      const float4 u4 = *reinterpret_cast<const float4*>(sU + r * NT + ((tj ^ (r & GM)) * 4));
      const float ri = cur.ri;
      const float rinv = 1.f / ri;
      const float uv[4] = {u4.x, u4.y, u4.z, u4.w};
      float pn[4], xn[4], rn[4];
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        // the step of passH: p = z + beta p, q = HA T/(N-1) + r_i p, x += alpha p, r -= alpha q
        const float uu = uv[y] * tsi[y];
        const float zz = PC ? cur.rr[y] * rinv : cur.rr[y];
        pn[y] = be[y] == 0.f ? zz : fmaf(be[y], cur.pp[y], zz);
        const float qq = fmaf(ri, pn[y], uu);
        xn[y] = fmaf(al[y], pn[y], cur.xx[y]);
        rn[y] = fmaf(-al[y], qq, cur.rr[y]);
        const float zn = PC ? rn[y] * rinv : rn[y];
        const bool live = valid && j0 + y < N;
        if (live) {
          s1[y] = fmaf(rn[y], zn, s1[y]);
          s2[y] = fmaf(rn[y], rn[y], s2[y]);
          s3[y] = fmaf(ri * zn, zn, s3[y]);
          s4[y] = fmaf(ri * zn, pn[y], s4[y]);
        }
        const float zv = live ? zn * zsc[y] : 0.f;
        const T16 zh = H16<T16>::from(zv);
        *bg_ptr(0, j0 + y, r) = zh;
        if (SPLIT) *bg_ptr(1, j0 + y, r) = H16<T16>::from(zv - (float)zh);
      }
      if (valid) {
        st4<float>(P + i * N, j0, N, vec, pn);
        st4<float>(X + i * N, j0, N, vec, xn);
        st4<float>(Res + i * N, j0, N, vec, rn);
      }
    }
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      // B = the same tile image read MN-major: K = rows (row-group stride sbo_u, two per K
      // block of 16), N = NT (core stride 128 B)
      const uint32_t au = smem_addr(sAu(q)), bg = smem_addr(sBg);
      // split operands: the cross terms of the tile first, then hi*hi
      if (SPLIT) {
#pragma unroll
        for (int kb = 0; kb < kTR / 16; ++kb) {
          const uint64_t A0 = umma_desc(bg + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
          const uint64_t B0 = umma_desc(au + kb * 2 * sbo_u, sbo_u, 128);
          const uint64_t A1 = umma_desc(bg + L::BGP + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
          const uint64_t B1 = umma_desc(au + L::AU * 2 + kb * 2 * sbo_u, sbo_u, 128);
          umma_f16(d_g, A0, B1, idesc_g, kb == 0 ? 0u : 1u);
          umma_f16(d_g, A1, B0, idesc_g, 1u);
        }
      }
#pragma unroll
      for (int kb = 0; kb < kTR / 16; ++kb) {
        const uint64_t A0 = umma_desc(bg + kb * 2 * L::LBOG, L::LBOG, L::SBOG);
        const uint64_t B0 = umma_desc(au + kb * 2 * sbo_u, sbo_u, 128);
        umma_f16(d_g, A0, B0, idesc_g, (kb == 0 && !SPLIT) ? 0u : 1u);
      }
      umma_commit(mbar_g);
    }
  }
  // the last tile's Gram
  if (Qb > 0) {
    if (!mbar_wait(mbar_g, ph_g, status)) ok = false;
    ph_g ^= 1u;
    tc_fence_after();
    gram_out();
  }
  tc_cp_wait_all();
  // the pass's partial Gram: row j, column k -> out[k*N + j] / zs_j (all zero when Qb == 0);
  // with atomic_out it is added into the FP32 total at reinterpret_cast<float*>(out)[k*N + j]
  // (the layout in which reduce_slice leaves the reduced Gram) instead
  if (g_owner && rt < N) {
    const float inv = gsi / zs[rt];
    for (int k = half * HALF; k < half * HALF + HALF; ++k)
      if (k < N) {
        const float v = sG[rt * (NT + 1) + k] * inv;
        if (atomic_out) atomicAdd(reinterpret_cast<float*>(out) + k * N + rt, v);
        else out[k * N + rt] = (double)v;
      }
  }
  tc_fence_before();
  __syncthreads();
  // column sums [(r, z) | (r, r) | sum r_i z^2 | sum r_i z p]: the RI row sweeps of each
  // column, in a fixed order (the z region is free)
  double* red = reinterpret_cast<double*>(sBg);
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    red[(0 * RI + ti) * NT + j0 + y] = (double)s1[y];
    red[(1 * RI + ti) * NT + j0 + y] = (double)s2[y];
    red[(2 * RI + ti) * NT + j0 + y] = (double)s3[y];
    red[(3 * RI + ti) * NT + j0 + y] = (double)s4[y];
  }
  __syncthreads();
  if (t < N) {
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double a = 0.0;
      for (int qq = 0; qq < RI; ++qq) a += red[(cc * RI + qq) * NT + t];
      if (atomic_out) atomicAdd(out + N * N + cc * N + t, a);
      else out[N * N + cc * N + t] = a;
    }
  }
  __syncthreads();
}

// The power of two that scales the largest |HA| (hamax: its float bits) into [2^13, 2^14), so
// that the FP16 image neither overflows (65,504) nor loses its small entries to the subnormal
// range whatever the units of the state; 1 when there is no maximum. The passes undo it
// exactly (image_scale_inv).
__device__ __forceinline__ float image_scale(const unsigned* hamax) {
  const float mx = hamax ? __uint_as_float(*hamax) : 0.f;
  if (!(mx > 0.f) || !isfinite(mx)) return 1.f;
  int e;
  frexpf(mx, &e);   // mx = f 2^e, f in [1/2, 1)
  return ldexpf(1.f, 14 - e);
}
__device__ __forceinline__ float image_scale_inv(const unsigned* hamax) { return 1.f / image_scale(hamax); }

// The tile images of the tensor-core pass, from the double-float HA: for CTA b (rows
// [b rows_per, ...)) and its tile q (128 rows), at (b qmax + q) TM 128 NT elements: [hi | lo],
// element (r, k) of each part at core_idx(r, k, NT); hi = round(HA), lo = round(HA - hi) in
// T16. Entries outside [0, m) x [0, N) are never written (the buffer is zeroed once when the
// handle is created).
template <typename T16, int TERMS>
__global__ void tc_images_kernel(const df32* __restrict__ HAdf, int64_t m, int N, int NT, int64_t rows_per,
                                 int qmax, T16* __restrict__ img, const unsigned* __restrict__ hamax) {
  constexpr int TM = TERMS == 3 ? 2 : 1;
  const int64_t tile = (int64_t)TM * kTR * NT;
  const float sc = image_scale(hamax);   // exact power of two
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m * N; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    const int64_t b = i / rows_per, l = i - b * rows_per;
    const int q = (int)(l / kTR), r = (int)(l % kTR);
    T16* base = img + (b * qmax + q) * tile;
    const df32 h = HAdf[e];
    const float hs = h.hi * sc;
    const T16 hi = H16<T16>::from(hs);
    base[core_idx(r, k, NT)] = hi;
    if (TM == 2) base[(int64_t)kTR * NT + core_idx(r, k, NT)] = H16<T16>::from((hs - (float)hi) + h.lo * sc);
  }
}

// Stage T^T/(N-1) scaled per column (ts_j = 1/rms_k(T_kj/(N-1))) into the B operand of the
// u MMA (rows j, K-major over k); also the column norms ||T_:j||^2 in FP64. T arrives in FP32
// (reduce_slice's FP32 output): the norms are exact-product compensated sums of the FP32
// values, and the scaling and the hi/lo split are FP32 (lo = v - hi is exact in FP32), so no
// per-entry FP64 arithmetic runs in any CTA.
template <typename T16, int NT, int TERMS>
__device__ __forceinline__ void stage_Tt16(const double* __restrict__ Tred, int N, double inv,
                                           T16* sBu, float* ts, double* tn2, double* scratch) {
  constexpr int L = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, k0 = t / NT;
  const float* T32 = reinterpret_cast<const float*>(Tred);
  SqAcc acc;
  for (int k = k0; k < NT; k += L) acc.add((k < N && j < N) ? __ldcg(T32 + k * N + j) : 0.f);
  scratch[t] = acc.value();
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < L; ++q) s += scratch[q * NT + t];
    tn2[t] = s;
    const double rms = sqrt(s / (double)(N > 0 ? N : 1)) * inv;
    ts[t] = (t < N && rms > 0.0) ? (float)(1.0 / rms) : 1.f;
    ts[NT + t] = (t < N && rms > 0.0) ? (float)rms : 1.f;   // 1/ts: undoes the scale on u
  }
  __syncthreads();
  const float inv_f = (float)inv;
  for (int e = t; e < NT * NT; e += kThreads) {
    const int jj = e / NT, k = e % NT;
    const float v = (k < N && jj < N) ? __ldcg(T32 + k * N + jj) * inv_f * ts[jj] : 0.f;
    const T16 hi = H16<T16>::from(v);
    sBu[core_idx(jj, k, NT)] = hi;
    if (TERMS == 3) sBu[NT * NT + core_idx(jj, k, NT)] = H16<T16>::from(v - H16<T16>::to(hi));
  }
  fence_async_smem();
  __syncthreads();
}

// The recursive form of stage_Tt16 for the one-reduction Hestenes-Stiefel step (see passH in
// cg_device.cuh): T_{k+1} = Tz + beta_j T_k with Tz the reduced HA^T z_{k+1} (FP32 at the
// start of Tred); T_k is not read where beta_j = 0. For NT <= 64 every CTA keeps T_k in its
// own shared memory (sTk, FP32 [NT][NT]; each entry is read and written by the same thread);
// NT = 128 has no room for it, and T_k is read from the global copy Tprev while CTA 0 writes
// T_{k+1} to Tnext (a ping-pong pair; every CTA computes the same values in the same order).
// With `step`, beta_j = gamma_{k+1}/gamma_k is formed from the reduced column sums and the
// column's scalars are advanced as in stage_T_rec. Then the column norms (tn2, FP64 from
// compensated FP32 sums), the per-column scale ts = 2^-e (a power of two, so that the scaling
// and its undoing on u are exact; e from the column's RMS, computed in FP32) and the split B
// operand of the u MMA. Each thread owns pairs of consecutive k of one column j, so the two
// 16-bit values of a pair go to shared memory in one 32-bit store (they are adjacent in the
// core-matrix layout).
template <typename T16, int NT, int TERMS>
__device__ __noinline__ void stage_Tt16_rec(const double* __restrict__ Tred, int N, double inv, float usi, const float* Tprev,
                               float* Tnext, bool write_next, float* sTk, float* beta, bool step,
                               const int* s_active, double* s_sig, double* s_den, double* s_gam, int* s_iters,
                               T16* sBu, float* ts, double* tn2, double* scratch) {
  constexpr int L = kThreads / NT, KP = NT / (2 * L);   // pairs of k per thread
  const int t = threadIdx.x, j = t % NT, kp = t / NT;
  const float* T32 = reinterpret_cast<const float*>(Tred);
  float v[KP][2];
#pragma unroll
  for (int q = 0; q < KP; ++q)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * (kp + q * L) + h;
      v[q][h] = (k < N && j < N) ? __ldcg(T32 + k * N + j) : 0.f;
    }
  float bj = 0.f;
  double g1 = 0.0;
  const bool act = step && j < N && s_active[j];
  if (act) {
    g1 = __ldcg(Tred + N * N + j);
    bj = (float)(g1 / s_sig[j]);
  }
  SqAcc acc;
#pragma unroll
  for (int q = 0; q < KP; ++q)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * (kp + q * L) + h;
      if (bj != 0.f && k < N) v[q][h] = fmaf(bj, sTk ? sTk[k * NT + j] : __ldcg(Tprev + k * N + j), v[q][h]);
      if (sTk) sTk[k * NT + j] = v[q][h];
      else if (write_next && k < N && j < N) Tnext[k * N + j] = v[q][h];
      acc.add(v[q][h]);
    }
  scratch[t] = acc.value();
  __syncthreads();   // every read of s_sig above precedes the updates below
  if (t < NT) {
    double sum = 0.0;
    for (int q = 0; q < L; ++q) sum += scratch[q * NT + t];
    tn2[t] = sum;
    // ts = 2^(1 - e) with rms = f 2^e, f in [1/2, 1): the scaled column has RMS in [1, 2)
    const float rms = sqrtf((float)sum * (1.f / (float)(N > 0 ? N : 1))) * (float)inv;
    int e = 0;
    const bool live = t < N && rms > 0.f && isfinite(rms);
    if (live) frexpf(rms, &e);
    ts[t] = live ? ldexpf(1.f, 1 - e) : 1.f;
    ts[NT + t] = (live ? ldexpf(1.f, e - 1) : 1.f) * usi;   // undoes ts and the image scale on u
    if (step) {
      if (act) {
        const double g2 = __ldcg(Tred + N * N + N + t);
        const double g3 = __ldcg(Tred + N * N + 2 * N + t), g4 = __ldcg(Tred + N * N + 3 * N + t);
        const double be = g1 / s_sig[t];
        s_den[t] = g3 + 2.0 * be * g4 + be * be * s_den[t];
        s_sig[t] = g1;
        s_gam[t] = g2;
        s_iters[t] += 1;
      }
      beta[t] = bj;
    }
  }
  __syncthreads();
  const float inv_f = (float)inv;
  const float tsj = ts[j];
#pragma unroll
  for (int q = 0; q < KP; ++q) {
    const int k = 2 * (kp + q * L);
    const float x0 = v[q][0] * inv_f * tsj, x1 = v[q][1] * inv_f * tsj;
    const T16 h0 = H16<T16>::from(x0), h1 = H16<T16>::from(x1);
    *reinterpret_cast<uint32_t*>(sBu + core_idx(j, k, NT)) = pack16(h0, h1);
    if (TERMS == 3)
      *reinterpret_cast<uint32_t*>(sBu + NT * NT + core_idx(j, k, NT)) =
          pack16(H16<T16>::from(x0 - H16<T16>::to(h0)), H16<T16>::from(x1 - H16<T16>::to(h1)));
  }
  fence_async_smem();
  __syncthreads();
}

struct MixedParams {
  int64_t m;
  int N;
  const void* HA16;   // tile images of HA (tc_images_kernel)
  int qmax;           // tiles per CTA row block in the images
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
  float* Tk;        // [2][N][N] the recursively updated T of the step (written by CTA 0)
  const unsigned* hamax;   // largest |HA| (float bits): the images' power-of-two scale
  float zr;   // PC: power of two nearest the typical r_i (z = R^-1 r is about r / zr)
  double* Tacc;     // [3][N N + 4 N] step totals accumulated by atomic adds (atomic_reduce)
  int atomic_reduce;   // N <= 64: a step's sums are added into Tacc (one barrier per step)
  double tol, inner_tol, itol_floor;
  int max_iter, refresh_every;
  int* col_iters;
  double* col_relres;
  double* col_true;
  int* status;
  unsigned* bar;
  unsigned long long* prof;   // optional phase timers of CTA 0 (ns), nullptr when off
};

template <typename T16, int NT, bool PC, int TERMS>
__global__ void __launch_bounds__(kThreads, 1) solve_mixed_kernel(MixedParams p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[4];   // u (NT = 128), Gram, u slots 0 and 1 (NT <= 64)
  __shared__ uint32_t tmem_base;
  double* s_gam = reinterpret_cast<double*>(smem);
  double* s_gold = s_gam + NT;
  double* s_sig = s_gold + NT;
  double* s_tn2 = s_sig + NT;
  double* s_bn2 = s_tn2 + NT;
  double* s_dn2 = s_bn2 + NT;
  double* s_alpha = s_dn2 + NT;
  double* s_den = s_alpha + NT;   // the previous step's Chronopoulos-Gear denominator
  double* s_prev = s_den + NT;
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
  // tensor-core operands (inside the union; the refresh passes reuse the same bytes)
  using TL = TcLayout<NT, TERMS>;
  T16* sBu = reinterpret_cast<T16*>(uni + TL::off_bu);
  float* s_zs = reinterpret_cast<float*>(uni + TL::off_zs);
  float* s_ts = reinterpret_cast<float*>(uni + TL::off_ts);
  float* sTk = TL::DB ? reinterpret_cast<float*>(uni + TL::off_tk) : nullptr;

  const int N = p.N, G = gridDim.x, b = blockIdx.x, t = threadIdx.x, warp = t >> 5;
  const int64_t rows_per = (p.m + G - 1) / G;
  const int64_t row0 = imin64(p.m, (int64_t)b * rows_per);
  const int64_t row1 = imin64(p.m, row0 + rows_per);
  const int NE = N * N + 4 * N;   // [N x N Gram | four N-vectors of column sums]
  GridBarrier bar{p.bar, reinterpret_cast<int*>(p.bar + 1), p.status, (unsigned)G, 0u};
  const double inv_nm1 = 1.0 / (double)(N - 1);
  double* Tp = p.Tpart + (int64_t)b * NE;
  // this CTA's tile images (tc_images_kernel uses the same row blocks)
  const T16* img = static_cast<const T16*>(p.HA16) + (size_t)b * p.qmax * TL::TILE;
  constexpr int TMC = tc_tmem_cols<NT>();

  if (t == 0) { mbar_init(&mbar[0]); mbar_init(&mbar[1]); mbar_init(&mbar[2]); mbar_init(&mbar[3]); }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)), "r"(TMC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  uint32_t ph_u = 0, ph_g = 0;
  uint32_t ph_u2[2] = {0u, 0u};
  int par = 0;
  bool ok = true;
  // atomic_reduce: CG steps so far (the same in every CTA) pick the step's accumulator; all
  // three start at zero (ordered before their first use by the first grid barrier)
  const bool atomic = NT <= 64 && p.atomic_reduce;
  const float img_si = image_scale_inv(p.hamax);   // undoes the images' scale (exact)
  int gstep = 0;
  if (atomic) {
    const int chunk = (3 * NE + G - 1) / G;
    const int e1 = min(3 * NE, (b + 1) * chunk);
    for (int e = b * chunk + t; e < e1; e += kThreads) p.Tacc[e] = 0.0;
  }
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
    // ---- inner solve of S X = B from X = 0 in the one-reduction Hestenes-Stiefel form: the
    // first reduction gives [HA^T z_0 | sum r_i z_0^2 | (r_0, r_0)], T_0 = HA^T z_0
    {
      ProSetup<float, PC> pro{p.B, p.X, p.Res, p.r32, N};
      passA<float, NT, ProSetup<float, PC>, PC>(p.HA32, row0, row1, N, p.r32, true, pro, uni, Tp);
    }
    if (t < N) {
      Tp[N * N + 2 * N + t] = 0.0;
      Tp[N * N + 3 * N + t] = 0.0;
    }
    if (!(ok = bar.sync())) break;
    reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, N * N);
    if (!(ok = bar.sync())) break;
    int tbuf = 0;   // the global copy of T_k the next staging reads
    stage_Tt16_rec<T16, NT, TERMS>(p.Tred, N, inv_nm1, img_si, p.Tk, p.Tk, b == 0, sTk, s_beta_v, false, s_active, s_sig,
                                   s_den, s_gam, s_iters, sBu, s_ts, s_tn2, scratch);
    if (t < NT) {
      const double sg = t < N ? __ldcg(p.Tred + N * N + t) : 0.0;       // sum r_i z_0^2
      const double gm = t < N ? __ldcg(p.Tred + N * N + N + t) : 0.0;   // (r_0, r_0)
      s_sig[t] = PC ? sg : gm;   // gamma = (r, z)
      s_den[t] = sg;             // sum r_i p^2
      s_beta_v[t] = 0.f;         // the first step takes p = z
      s_gam[t] = gm;
      s_bn2[t] = gm;   // residual norm^2 at the start of this inner solve
      s_active[t] = (t < N && !s_done[t] && gm > 0.0) ? 1 : 0;
    }
    __syncthreads();
    tick(PH_SETUP);
    int it = 0;
    for (;;) {
      int my_active = 0;
      if (t < NT) {
        int a = s_active[t];
        const double gm = s_gam[t];
        double al = 0.0;
        if (a && !isfinite(gm)) { atomicOr(p.status, DS_NONFINITE); a = 0; }
        // the inner solve of this column ends once its residual fell by the factor s_itol
        // (compared in squares: FP64 square roots are costly on this part's FP64 pipe)
        if (a && it > 0) {
          const double itf = (double)s_itol[t];
          if (gm <= itf * itf * s_bn2[t]) a = 0;
        }
        if (a) {
          // alpha = gamma / (p, S p), (p, S p) = ||T||^2/(N-1) + sum r_i p^2; a non-positive or
          // non-finite value means the low-precision recurrences have drifted: this column's
          // inner solve ends here and the refresh restarts it
          const double pq = s_tn2[t] * inv_nm1 + s_den[t];
          if (!isfinite(pq) || !(pq > 0.0)) a = 0;
          else al = s_sig[t] / pq;
        }
        s_active[t] = a;
        s_alpha[t] = al;
        s_alpha_v[t] = (float)al;
        // the Gram's z operand scaled to unit norm: z = r (or R^-1 r, about r / zr) over ||r||,
        // whatever the units of the problem
        s_zs[t] = (t < N && gm > 0.0) ? (float)(1.0 / sqrt(gm)) * (PC ? p.zr : 1.f) : 1.f;
        my_active = a;
      }
      const int any = __syncthreads_or(my_active);
      if (!(any && (p.refresh_every <= 0 || it < p.refresh_every) && total + it < p.max_iter)) break;
      tick(PH_SCAL);
      // the step's sums: into this CTA's partial (then a fixed-order reduction between two grid
      // barriers), or added into the step's accumulator (atomic_reduce: one barrier; the
      // accumulator two steps ahead is cleared behind it, every CTA having read it before)
      double* acc = atomic ? p.Tacc + (size_t)(gstep % 3) * NE : Tp;
      if constexpr (NT <= 64)
        passF_tc_db<T16, NT, PC, TERMS>(img, row0, row1, N, p.X, p.Res, p.P, p.r32, s_alpha_v,
                                        s_beta_v, uni, tmem, &mbar[2], &mbar[1], ph_u2, ph_g, p.status, ok, acc,
                                        atomic, img_si);
      else
        passF_tc2<T16, NT, PC, TERMS>(img, p.qmax, row0, row1, N, p.X, p.Res, p.P, p.r32, s_alpha_v,
                                      s_beta_v, uni, tmem, &mbar[0], &mbar[1], ph_u, ph_g, p.status, ok, Tp, img_si);
      tick(PH_PASS);
      if (!(ok = bar.sync() && ok)) break;
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
        reduce_slice(p.Tpart, G, NE, p.Tred, scratch, b, N * N);
        tick(PH_RED);
        if (!(ok = bar.sync())) break;
        tick(PH_BAR2);
      }
      // beta, T_{k+1} = HA^T z_{k+1} + beta T_k (from the global copy of T_k), the scalars
      const float* Tprev = p.Tk + (size_t)tbuf * N * N;
      float* Tnext = p.Tk + (size_t)(tbuf ^ 1) * N * N;
      stage_Tt16_rec<T16, NT, TERMS>(tsum, N, inv_nm1, img_si, Tprev, Tnext, b == 0, sTk, s_beta_v, true, s_active,
                                     s_sig, s_den, s_gam, s_iters, sBu, s_ts, s_tn2, scratch);
      tbuf ^= 1;
      ++it;
      tick(PH_SCAL);
    }
    if (!ok) break;
    total += it;
    ++cycles;
    // ---- double-float refresh: Z += X; T = HA^T Z; W; true residual D - S Z -> next B
    if ((N & 3) == 0) {
      refreshA_async<NT>(p.HAdf, p.Zdf, p.X, row0, row1, N, uni, Tp);
    } else {
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
      bool done_b = false;
      if constexpr (DFTile<NT>::B_ASYNC) {
        if ((N & 3) == 0) {
          refreshB_async<NT, float>(p.HAdf, p.Zdf, p.Ddf, p.r, p.B, row0, row1, N, sTd, df32(inv_nm1),
                                    uni + NT * LDD * sizeof(df32), s_tmp);
          done_b = true;
        }
      }
      if (!done_b) {
        EpiRefreshDF<float> epi{p.Zdf, p.Ddf, p.r, p.B, N, df32(inv_nm1)};
        passB<df32, NT>(p.HAdf, row0, row1, N, sTd, uni + NT * LDD * sizeof(df32), epi, s_tmp);
      }
    }
    if (t < NT) p.rrpart[((int64_t)par * G + b) * NT + t] = s_tmp[t];
    if (!(ok = bar.sync())) break;
    reduce_all<NT>(p.rrpart + (int64_t)par * G * NT, G, N, s_tmp, scratch);
    par ^= 1;
    if (t < N) {
      // a non-finite residual or ||d_j|| (NaN or Inf in the inputs) ends the column with the
      // non-finite status
      const bool fin = isfinite(s_dn2[t]) && isfinite(s_tmp[t]);
      if (!fin) atomicOr(p.status, DS_NONFINITE);
      const double rel = !fin ? (double)NAN : (s_dn2[t] > 0.0 ? sqrt(s_tmp[t] / s_dn2[t]) : 0.0);
      s_rel[t] = rel;
      s_true[t] = rel;
      if (!s_done[t]) {
        // converged, stalled (no halving over a cycle) or non-finite
        if (!fin || rel <= p.tol || (cycles >= 2 && rel > 0.5 * s_prev[t])) s_done[t] = 1;
      }
      s_prev[t] = rel;
      // the next inner solve only has to gain the remaining factor tol/rel (margin 0.1),
      // but not more than the low-precision operator allows
      double it_next = rel > 0.0 ? 0.1 * p.tol / rel : 0.5;
      it_next = fmax(it_next, fmax(p.inner_tol, p.itol_floor));
      s_itol[t] = (float)fmin(it_next, 0.5);
    }
    const int all_done = __syncthreads_and(t >= N || s_done[t]);
    tick(PH_REFRESH);
    // every cycle either takes a step (total grows to at most max_iter) or ends the solve:
    // without an active column (it == 0) the next cycle would repeat this one
    if (all_done || total >= p.max_iter || it == 0) break;
  }

  if (prof)
    for (int q = 0; q < PH_COUNT; ++q) p.prof[q] = ph[q];
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
  constexpr int tcb0 = TcLayout<NT, TERMS>::bytes;
  constexpr int tcb = tcb0 > DFTile<NT>::bytes ? tcb0 : DFTile<NT>::bytes;
  constexpr int u = refresh_union_bytes<NT>() > tcb ? refresh_union_bytes<NT>() : tcb;
  return scalar_bytes<NT>() + kThreads * 8 + u;
}

}  // namespace enkf
