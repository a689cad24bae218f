// The ensemble update X_a = X_f + A W (Fig. 2, Algorithm 1: A = X_f - xbar 1^T, W = HA^T Z/(N-1))
// on the 5th-generation tensor cores, for FP32 ensembles.
//
// Per 128-row tile of X_f: the rows are staged in shared memory (16-byte cp.async; for N <= 64
// the next two tiles' copies are in flight behind the current one), each row's mean and largest anomaly are
// formed, and the anomalies scaled by an exact power of two per row (so FP16 neither overflows
// nor flushes) are split into hi + lo FP16 parts in the canonical K-major core-matrix layout,
// the lo part stored times 2^11 so that it stays in FP16's normal range. W is staged once per
// CTA the same way (rows j, K-major over k, a power-of-two scale per column). D = A W runs as
// three M = 128 x N = NT x K = NT MMAs per K block with FP32 accumulation in TMEM: hi*hi into
// one accumulator, hi*lo' + lo'*hi into a second, so D = D1 + 2^-11 D2 carries about 22
// significant bits per product; the epilogue reads both row by row, undoes the scales, forms
// X_a = X_f + D in place of the staged tile and then writes the tile out with coalesced
// 16-byte stores (a row per thread would scatter every store over 32 rows). X_a may be
// X_f itself: a tile is read into shared memory before any of its rows is written, and no CTA
// reads another CTA's tiles.
#include <algorithm>
#include <cmath>

#include "tc_mixed.cuh"

namespace enkf {

template <int NT> struct UpdLayout {
  static constexpr int LDX = NT + 4;                       // staged X_f row stride (floats)
  static constexpr int XT = kTR * LDX * 4;                 // bytes per staged tile
  static constexpr int AIMG = 2 * kTR * NT * 2;            // A image: hi and lo parts
  static constexpr int BIMG = 2 * NT * NT * 2;             // W image: hi and lo parts
  static constexpr int NBUF = NT <= 64 ? 3 : 1;            // staged tiles (NT = 128: one, smem)
  static constexpr int off_x = 0;
  static constexpr int off_a = ((NBUF * XT + 1023) / 1024) * 1024;
  static constexpr int off_b = off_a + AIMG;
  static constexpr int off_rs = off_b + BIMG;              // per-row 2^-e scale [128]
  static constexpr int off_mean = off_rs + 4 * kTR;        // per-row mean [128]
  static constexpr int off_ws = off_mean + 4 * kTR;        // per-column 1/scale of W [NT]
  static constexpr int bytes = off_ws + 4 * NT;
  static_assert(off_a % 1024 == 0 && off_b % 1024 == 0, "operand alignment");
};
template <int NT> __host__ __device__ constexpr int update_tc_smem_bytes() { return UpdLayout<NT>::bytes; }

// 2^-e with 2^e >= max|v| > 2^(e-1) (1 for v = 0): scales v into (1/2, 1] exactly
__device__ __forceinline__ float pow2_scale(float vmax) {
  if (!(vmax > 0.f) || !isfinite(vmax)) return 1.f;
  int e;
  frexpf(vmax, &e);
  return ldexpf(1.f, -e);
}

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) update_tc_kernel(const float* Xf, float* Xa,
                                                                const double* __restrict__ W, int64_t n,
                                                                int N, int* status) {
  using L = UpdLayout<NT>;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  constexpr int TMC = 2 * NT;   // D1 (hi*hi) at column 0, D2 (the cross terms) at column NT
  constexpr uint32_t idesc = umma_idesc(H16<__half>::fmt, NT);
  constexpr uint32_t sbo = (NT / 8) * 128;
  constexpr int C4 = NT / 4, HALF = NT / 2, CH = HALF / 16;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, qd = warp & 3, half = warp >> 2;
  float* sX0 = reinterpret_cast<float*>(smem + L::off_x);
  __half* sA = reinterpret_cast<__half*>(smem + L::off_a);
  __half* sB = reinterpret_cast<__half*>(smem + L::off_b);
  float* s_rs = reinterpret_cast<float*>(smem + L::off_rs);
  float* s_mean = reinterpret_cast<float*>(smem + L::off_mean);
  float* s_ws = reinterpret_cast<float*>(smem + L::off_ws);
  if (dynamic_smem_bytes() < (unsigned)L::bytes) {
    if (t == 0) atomicOr(status, DS_SMEM);
    return;
  }
  if (t == 0) mbar_init(&mbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)), "r"(TMC));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // W: per-column power-of-two scale, then the hi/lo image (rows j, K-major over k)
  if (t < NT) {
    float mx = 0.f;
    if (t < N)
      for (int k = 0; k < N; ++k) mx = fmaxf(mx, fabsf((float)__ldcg(W + k * N + t)));
    const float sc = pow2_scale(mx);
    s_ws[t] = 1.f / sc;                                   // exact (a power of two)
    for (int k = 0; k < NT; ++k) {
      const float v = (t < N && k < N) ? (float)__ldcg(W + k * N + t) * sc : 0.f;
      const __half hi = __float2half_rn(v);
      sB[core_idx(t, k, NT)] = hi;
      sB[NT * NT + core_idx(t, k, NT)] = __float2half_rn((v - __half2float(hi)) * 2048.f);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const bool vec = (N & 3) == 0;
  const int64_t ntiles = (n + kTR - 1) / kTR;
  auto stage = [&](int64_t tile, float* sX) {
    const int64_t i0 = tile * kTR;
    for (int c = t; c < kTR * C4; c += kThreads) {
      const int r = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + r;
      const bool ok = i < n && c0 < N;
      if (vec) {
        cp_async16(sX + r * L::LDX + c0, ok ? Xf + i * N + c0 : Xf, ok);
      } else {
        float a[4] = {0.f, 0.f, 0.f, 0.f};
        if (ok) ld4<float>(a, Xf + i * N, c0, N, false);
        *reinterpret_cast<float4*>(sX + r * L::LDX + c0) = make_float4(a[0], a[1], a[2], a[3]);
      }
    }
    cp_async_commit();
  };
  uint32_t ph = 0;
  bool ok = true;
  auto xbuf = [&](int64_t k) { return sX0 + (int)(k % L::NBUF) * (L::XT / 4); };
  // NBUF - 1 tiles in flight ahead of the one being processed (one commit group per tile,
  // empty past the end, so that "all but the newest NBUF - 1 groups" is always this tile)
  if (L::NBUF > 1)
    for (int q = 0; q < L::NBUF - 1; ++q) {
      const int64_t tq = (int64_t)blockIdx.x + (int64_t)q * gridDim.x;
      if (tq < ntiles) stage(tq, xbuf(q));
      else cp_async_commit();
    }
  int64_t k = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++k) {
    float* sX = xbuf(k);
    if (L::NBUF == 1) {
      stage(tile, sX);
      cp_async_wait<0>();
    } else {
      const int64_t nxt = tile + (int64_t)(L::NBUF - 1) * gridDim.x;
      if (nxt < ntiles) stage(nxt, xbuf(k + L::NBUF - 1));   // the buffer of tile k - 1, consumed
      else cp_async_commit();
      cp_async_wait<(L::NBUF > 1 ? L::NBUF - 1 : 0)>();
    }
    __syncthreads();
    // row means and the largest anomaly of each row: two threads per row
    {
      const int r = t >> 1, hf = t & 1;
      float sum = 0.f;
      for (int k = hf; k < N; k += 2) sum += sX[r * L::LDX + k];
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      const float mean = sum / (float)N;
      float mx = 0.f;
      for (int k = hf; k < N; k += 2) mx = fmaxf(mx, fabsf(sX[r * L::LDX + k] - mean));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
      const float sc = pow2_scale(mx);
      if (hf == 0) {
        s_mean[r] = mean;
        s_rs[r] = sc;
      }
      // the scaled anomalies as hi + lo FP16, 8 consecutive k (one 16-byte core row) at a time
      for (int kc = hf; kc < NT / 8; kc += 2) {
        __align__(16) __half hv[8], lv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = kc * 8 + e;
          const float a = k < N ? (sX[r * L::LDX + k] - mean) * sc : 0.f;
          hv[e] = __float2half_rn(a);
          lv[e] = __float2half_rn((a - __half2float(hv[e])) * 2048.f);
        }
        *reinterpret_cast<uint4*>(sA + core_idx(r, kc * 8, NT)) = *reinterpret_cast<const uint4*>(hv);
        *reinterpret_cast<uint4*>(sA + kTR * NT + core_idx(r, kc * 8, NT)) = *reinterpret_cast<const uint4*>(lv);
      }
    }
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t au = smem_addr(sA), bu = smem_addr(sB);
#pragma unroll
      for (int kb = 0; kb < NT / 16; ++kb) {
        umma_f16(tmem, umma_desc(au + kb * 256, 128, sbo), umma_desc(bu + kb * 256, 128, sbo), idesc, kb > 0 ? 1u : 0u);
        umma_f16(tmem + NT, umma_desc(au + kb * 256, 128, sbo), umma_desc(bu + 2 * NT * NT + kb * 256, 128, sbo), idesc,
                 kb > 0 ? 1u : 0u);
        umma_f16(tmem + NT, umma_desc(au + 2 * kTR * NT + kb * 256, 128, sbo), umma_desc(bu + kb * 256, 128, sbo), idesc, 1u);
      }
      umma_commit(&mbar);
    }
    if (!mbar_wait(&mbar, ph, status)) ok = false;
    ph ^= 1u;
    tc_fence_after();
    // X_a = X_f + D / (row scale * column scale), one row per thread (TMEM lane = row)
    const int rt = 32 * qd + lane;
    const int64_t i = tile * kTR + rt;
    const float irs = 1.f / s_rs[rt];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int j0 = half * HALF + 16 * c;
      float d[16], d2[16];
      tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + j0, d);
      tmem_ld16(tmem + ((uint32_t)(32 * qd) << 16) + NT + j0, d2);
#pragma unroll
      for (int y = 0; y < 16; ++y) d[y] = fmaf(d2[y], 0x1p-11f, d[y]);
      if (i < n) {
#pragma unroll
        for (int y4 = 0; y4 < 4; ++y4) {
          const int jj = j0 + 4 * y4;
          if (jj < N) {
            float* xr = sX + rt * L::LDX + jj;
            const float4 xf = *reinterpret_cast<const float4*>(xr);
            *reinterpret_cast<float4*>(xr) = make_float4(fmaf(d[4 * y4] * irs, s_ws[jj], xf.x),
                                                         fmaf(d[4 * y4 + 1] * irs, s_ws[jj + 1], xf.y),
                                                         fmaf(d[4 * y4 + 2] * irs, s_ws[jj + 2], xf.z),
                                                         fmaf(d[4 * y4 + 3] * irs, s_ws[jj + 3], xf.w));
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    // the finished tile out: consecutive threads on consecutive 16-byte pieces of a row
    for (int c = t; c < kTR * C4; c += kThreads) {
      const int r = c / C4, c0 = (c % C4) * 4;
      const int64_t ig = tile * kTR + r;
      if (ig < n && c0 < N) {
        const float4 v = *reinterpret_cast<const float4*>(sX + r * L::LDX + c0);
        const float o[4] = {v.x, v.y, v.z, v.w};
        st4<float>(Xa + ig * N, c0, N, vec, o);
      }
    }
    __syncthreads();   // the staged tile, the A image and TMEM are rewritten by the next tile
  }
  cp_async_wait<0>();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMC));
}

template <int NT>
static cudaError_t launch_one(const float* Xf, float* Xa, const double* W, int64_t n, int N, int* status,
                              int sms, cudaStream_t s) {
  constexpr int smem = update_tc_smem_bytes<NT>();
  cudaError_t e = cudaFuncSetAttribute(update_tc_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + kTR - 1) / kTR;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms));
  update_tc_kernel<NT><<<grid, kThreads, smem, s>>>(Xf, Xa, W, n, N, status);
  return cudaGetLastError();
}

// X_a = X_f + (X_f - xbar 1^T) W for FP32 ensembles on the tensor cores.
cudaError_t launch_update_tc(enkf_handle_s* h, const void* Xf, void* Xa) {
  const auto& c = h->cfg;
  const float* x = static_cast<const float*>(Xf);
  float* xa = static_cast<float*>(Xa);
  const int NT = c.N <= 32 ? 32 : (c.N <= 64 ? 64 : 128);
  if (NT == 32) return launch_one<32>(x, xa, h->ws.W, c.n, c.N, h->ws.status, h->sms, h->stream);
  if (NT == 64) return launch_one<64>(x, xa, h->ws.W, c.n, c.N, h->ws.status, h->sms, h->stream);
  return launch_one<128>(x, xa, h->ws.W, c.n, c.N, h->ws.status, h->sms, h->stream);
}

}  // namespace enkf
