// The row-range form of the innovation step (Algorithm 1: Zobs = H X_f, HA = Zobs - zbar 1^T,
// D = y 1^T + E - Zobs) with the observation perturbations E drawn from Philox4x32-10 and
// Box-Muller: shared by the single-analysis innovations kernel (kernels_fp.cu) and the batched
// kernel (kernels_batch.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cg_device.cuh"

namespace enkf {

// ------------------------------------------------------------------ K1: innovations
// Standard normals of members (j, j + 1), j even, from one Philox block and one Box-Muller
// pair (the definition of perturbation_normal for both members, computed once).
__device__ __forceinline__ void perturbation_pair(int64_t i, int j, uint64_t seed, uint64_t counter,
                                                  double& n_even, double& n_odd) {
  uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(j >> 1), c2 = (uint32_t)counter, c3 = (uint32_t)(counter >> 32);
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t x1 = ((uint64_t)c0 << 21) | (c1 >> 11);
  const uint64_t x2 = ((uint64_t)c2 << 21) | (c3 >> 11);
  const double u1 = ((double)x1 + 0.5) * 0x1p-53;
  const double u2 = (double)x2 * 0x1p-53;
  const double rho = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincos(6.283185307179586 * u2, &sn, &cs);
  n_even = rho * cs;
  n_odd = rho * sn;
}

// The same pair in single precision, for the modes that compute in FP32 (FP32 and the
// tensor-core modes): the same Philox block and the same 53-bit uniforms u1 = (x1 + 1/2)
// 2^-53 and u2 = x2 2^-53, rounded to float, with float log (log1p of -(1 - u1) when
// u1 >= 1/2, where 1 - u1 is formed exactly from the integer), square root and sin/cos of
// pi 2 u2. Each normal is within about 1e-7 (relative to its size) of the FP64 form, and the
// FP64 log and sincos, which dominate the innovations on a GPU whose FP64 rate is a small
// fraction of its FP32 rate, are avoided.
// Conversions that stay off the FP64 pipe (two operations per clock per SM on this part; the
// 64-bit conversion instructions run there too).
// The float nearest to the 53-bit integer a 2^21 + b (a < 2^32, b < 2^21), as a 64-bit to
// float conversion rounds it, from 32-bit conversions: for a >= 2^25 the rounding drops at
// least two bits of a, so ORing "b != 0" into its lowest bit supplies the sticky bit without
// touching the round bit; otherwise a >> 1 and ((a & 1) << 21) | b are exact floats and one
// FP32 fused multiply-add rounds their exact sum once.
__device__ __forceinline__ float u53_to_float(uint32_t a, uint32_t b) {
  if (a >= (1u << 25)) return __uint2float_rn(a | (b != 0u ? 1u : 0u)) * 0x1p21f;
  return fmaf(__uint2float_rn(a >> 1), 0x1p22f, __uint2float_rn(((a & 1u) << 21) | b));
}
// (double)x by exponent rebias and mantissa shift for normal x and zero; subnormals,
// infinities and NaN take the conversion instruction.
__device__ __forceinline__ double f2d_bits(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xFFu;
  if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)((uint64_t)u << 32));
  if (e == 0u || e == 0xFFu) return (double)x;
  return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                                          ((uint64_t)(u & 0x7FFFFFu) << 29)));
}
// hi + lo rounded to FP64, as (double)hi + (double)lo: one FP64 addition
__device__ __forceinline__ double df_to_double(const df32& v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }
// df32(x) for a double x: hi = x rounded to float, lo = (x - hi) rounded to float, with the
// widening of hi done by f2d_bits (three FP64-pipe operations instead of four)
__device__ __forceinline__ df32 df_from_double(double x) {
  const float hi = __double2float_rn(x);
  return df32(hi, __double2float_rn(x - f2d_bits(hi)));
}

__device__ __forceinline__ void perturbation_pair_f32(int64_t i, int j, uint64_t seed, uint64_t counter,
                                                      float& n_even, float& n_odd) {
  uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(j >> 1), c2 = (uint32_t)counter, c3 = (uint32_t)(counter >> 32);
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t x1 = ((uint64_t)c0 << 21) | (c1 >> 11);
  float lg;
  if (x1 < (1ull << 52)) {
    lg = logf(fmaf(u53_to_float(c0, c1 >> 11), 0x1p-53f, 0x1p-54f));
  } else {
    const uint64_t y1 = (1ull << 53) - x1;   // 1 - u1 = (y1 - 1/2) 2^-53, y1 <= 2^52
    const float w = fmaf(u53_to_float((uint32_t)(y1 >> 21), (uint32_t)(y1 & 0x1FFFFFu)), 0x1p-53f, -0x1p-54f);
    lg = log1pf(-w);
  }
  const float rho = sqrtf(-2.f * lg);
  float sn, cs;
  sincospif(u53_to_float(c2, c3 >> 11) * 0x1p-52f, &sn, &cs);
  n_even = rho * cs;
  n_odd = rho * sn;
}
__device__ __forceinline__ void perturbation_pair_f32(int64_t i, int j, uint64_t seed, uint64_t counter,
                                                      double& n_even, double& n_odd) {
  float a, b;
  perturbation_pair_f32(i, j, seed, counter, a, b);
  n_even = (double)a;
  n_odd = (double)b;
}

// Rows [i_begin, i_end) of the observation operator, one warp per row: `warp` is this warp's
// index among `nwarps` warps sharing the range. Lane l owns members 2l, 2l + 1, 2l + 64,
// 2l + 65, so each perturbation pair is drawn once.
template <typename VT>
__device__ __forceinline__ void innov_rows_f64(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ HA64, float* __restrict__ HA32, double* __restrict__ D,
    float* __restrict__ B32, __nv_bfloat16* __restrict__ HAb, __half* __restrict__ HAh,
    int split_lo, df32* __restrict__ HAdf, df32* __restrict__ Ddf, int64_t i_begin, int64_t i_end,
    int64_t warp, int64_t nwarps) {
  // FP64 instructions are scarce on this part (2 per clock per SM): 1/N is applied as a
  // product and members 64..127 are skipped when N <= 64
  const int lane = threadIdx.x & 31;
  const double inv_n = 1.0 / (double)N;
  const bool wide = N > 64;   // members 64..127 present (warp-uniform)
  for (int64_t i = i_begin + warp; i < i_end; i += nwarps) {
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    const int k0 = rowptr[i], k1 = rowptr[i + 1];
    for (int k = k0; k < k1; ++k) {
      const double wk = w[k];
      const VT* xr = Xf + (int64_t)col[k] * N;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = 2 * lane + (q & 1) + 64 * (q >> 1);
        if (j < N) z[q] = fma(wk, (double)xr[j], z[q]);
      }
    }
    double s = z[0] + z[1];
    if (wide) s += z[2] + z[3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const double zbar = s * inv_n;
    const double yi = y[i], ri = r[i];
    const double sr = emode == 2 ? sqrt(ri) : 0.0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int jp = 2 * lane + 64 * h;   // even member of the pair
      if (jp >= N) continue;
      double nrm[2] = {0.0, 0.0};
      if (emode == 2) perturbation_pair(i, jp, seed, counter, nrm[0], nrm[1]);
      const int64_t e0 = i * N + jp;
      double hv[2], dv[2];
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        double pert = 0.0;
        if (jp + b < N) {
          if (emode == 1) pert = E[e0 + b];
          else if (emode == 2) pert = sr * nrm[b];
        }
        hv[b] = z[2 * h + b] - zbar;
        dv[b] = (yi - z[2 * h + b]) + pert;
      }
      if ((N & 1) == 0) {
        // both members present and e0 even: one 8- or 16-byte store per array per lane, so a
        // warp writes contiguous row segments
        if (HA64) *reinterpret_cast<double2*>(HA64 + e0) = make_double2(hv[0], hv[1]);
        *reinterpret_cast<double2*>(D + e0) = make_double2(dv[0], dv[1]);
        if (HA32) *reinterpret_cast<float2*>(HA32 + e0) = make_float2((float)hv[0], (float)hv[1]);
        if (B32) *reinterpret_cast<float2*>(B32 + e0) = make_float2((float)dv[0], (float)dv[1]);
        if (HAdf) {
          const df32 a0(hv[0]), a1(hv[1]);
          *reinterpret_cast<float4*>(HAdf + e0) = make_float4(a0.hi, a0.lo, a1.hi, a1.lo);
        }
        if (Ddf) {
          const df32 d0(dv[0]), d1(dv[1]);
          *reinterpret_cast<float4*>(Ddf + e0) = make_float4(d0.hi, d0.lo, d1.hi, d1.lo);
        }
      } else {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (jp + b >= N) continue;
          const int64_t e = e0 + b;
          if (HA64) HA64[e] = hv[b];
          D[e] = dv[b];
          if (HA32) HA32[e] = (float)hv[b];
          if (B32) B32[e] = (float)dv[b];
          if (HAdf) HAdf[e] = df32(hv[b]);
          if (Ddf) Ddf[e] = df32(dv[b]);
        }
      }
      // low-precision copies: hi part at [0, m N), lo part (ha - hi) at [m N, 2 m N) when split
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        if (jp + b >= N) continue;
        const int64_t e = e0 + b;
        const double ha = hv[b];
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

// The same rows for FP32 ensembles (the FP32 and tensor-core modes), in double-float (FP32
// pair) arithmetic: this part issues FP32 at 64x its FP64 rate, and the FP64 version spends
// its time in FP64 adds and FP32<->FP64 conversions. z = sum w_k x_k accumulates exact
// products of the double-float weight and the FP32 member value, z-bar is a double-float warp
// sum (each lane adds the same operands in the same order: the double-float sum is
// commutative), HA = z - z-bar and D = (y - z) + E are double-float (about 48 significant
// bits, the precision of the HAdf and Ddf arrays they fill), E = sqrt(r_i) times the FP32
// normal as an exact double-float product; HA32 and B32 are the high parts, and only the
// FP64 copy of D is widened per element.
template <typename VT>
__device__ __forceinline__ void innov_rows_df(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ HA64, float* __restrict__ HA32, double* __restrict__ D,
    float* __restrict__ B32, __nv_bfloat16* __restrict__ HAb, __half* __restrict__ HAh,
    int split_lo, df32* __restrict__ HAdf, df32* __restrict__ Ddf, int64_t i_begin, int64_t i_end,
    int64_t warp, int64_t nwarps, unsigned* hamax = nullptr) {
  static_assert(sizeof(VT) == 4, "double-float innovations take an FP32 ensemble");
  const int lane = threadIdx.x & 31;
  float hmax = 0.f;   // largest |HA| of the warp's rows (hamax: atomic maximum of the float bits)
  const df32 inv_n(1.0 / (double)N);
  const bool wide = N > 64;   // members 64..127 present (warp-uniform)
  // The warp's rows are i0 + q nwarps, q = 0, 1, ...; the per-row values that come from FP64
  // inputs (y_i, sqrt(r_i) and the weight of the row's first operator entry as double-float
  // pairs) are formed for 32 rows at a time, lane q for row i0 + q nwarps, and handed to the
  // other lanes by shuffles: one FP64 evaluation per row instead of one per lane.
  for (int64_t i0 = i_begin + warp; i0 < i_end; i0 += 32 * nwarps) {
    const int64_t il = i0 + (int64_t)lane * nwarps;
    df32 y_l, s_l, w_l;
    if (il < i_end) {
      y_l = df_from_double(y[il]);
      if (emode == 2) s_l = df_from_double(sqrt(r[il]));
      const int kf = rowptr[il];
      if (kf < rowptr[il + 1]) w_l = df_from_double(w[kf]);
    }
    for (int q32 = 0; q32 < 32; ++q32) {
      const int64_t i = i0 + (int64_t)q32 * nwarps;
      if (i >= i_end) break;   // warp-uniform
      const df32 yd(__shfl_sync(0xffffffffu, y_l.hi, q32), __shfl_sync(0xffffffffu, y_l.lo, q32));
      const df32 sr(__shfl_sync(0xffffffffu, s_l.hi, q32), __shfl_sync(0xffffffffu, s_l.lo, q32));
      const df32 w0(__shfl_sync(0xffffffffu, w_l.hi, q32), __shfl_sync(0xffffffffu, w_l.lo, q32));
      df32 z[4];
      const int k0 = rowptr[i], k1 = rowptr[i + 1];
      for (int k = k0; k < k1; ++k) {
        const df32 wk = k == k0 ? w0 : df_from_double(w[k]);
        const VT* xr = Xf + (int64_t)col[k] * N;
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = 2 * lane + (q & 1) + 64 * (q >> 1);
          if (j < N) z[q] = fma(wk, df32((float)xr[j], 0.f), z[q]);
        }
      }
      df32 s = z[0] + z[1];
      if (wide) s = s + (z[2] + z[3]);
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        s = s + df32(__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o));
      const df32 zbar = s * inv_n;
  #pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int jp = 2 * lane + 64 * h;   // even member of the pair
        if (jp >= N) continue;
        float nrm[2] = {0.f, 0.f};
        if (emode == 2) perturbation_pair_f32(i, jp, seed, counter, nrm[0], nrm[1]);
        const int64_t e0 = i * N + jp;
        df32 hv[2], dv[2];
  #pragma unroll
        for (int b = 0; b < 2; ++b) {
          df32 pert;
          if (jp + b < N) {
            if (emode == 1) pert = df_from_double(E[e0 + b]);
            else if (emode == 2) pert = sr * df32(nrm[b], 0.f);
          }
          hv[b] = z[2 * h + b] - zbar;
          dv[b] = (yd - z[2 * h + b]) + pert;
          if (jp + b < N) hmax = fmaxf(hmax, fabsf(hv[b].hi));
        }
        if ((N & 1) == 0) {
          // both members present and e0 even: one 8- or 16-byte store per array per lane
          *reinterpret_cast<double2*>(D + e0) = make_double2(df_to_double(dv[0]), df_to_double(dv[1]));
          if (HA32) *reinterpret_cast<float2*>(HA32 + e0) = make_float2(hv[0].hi, hv[1].hi);
          if (B32) *reinterpret_cast<float2*>(B32 + e0) = make_float2(dv[0].hi, dv[1].hi);
          if (HAdf) *reinterpret_cast<float4*>(HAdf + e0) = make_float4(hv[0].hi, hv[0].lo, hv[1].hi, hv[1].lo);
          if (Ddf) *reinterpret_cast<float4*>(Ddf + e0) = make_float4(dv[0].hi, dv[0].lo, dv[1].hi, dv[1].lo);
        } else {
  #pragma unroll
          for (int b = 0; b < 2; ++b) {
            if (jp + b >= N) continue;
            const int64_t e = e0 + b;
            D[e] = df_to_double(dv[b]);
            if (HA32) HA32[e] = hv[b].hi;
            if (B32) B32[e] = dv[b].hi;
            if (HAdf) HAdf[e] = hv[b];
            if (Ddf) Ddf[e] = dv[b];
          }
        }
        // optional copies (not requested by the current callers): FP64 HA and 16-bit images
  #pragma unroll
        for (int b = 0; b < 2; ++b) {
          if (jp + b >= N) continue;
          const int64_t e = e0 + b;
          if (HA64) HA64[e] = (double)hv[b];
          if (HAb) {
            const __nv_bfloat16 hi = __float2bfloat16(hv[b].hi);
            HAb[e] = hi;
            if (split_lo) HAb[m * N + e] = __float2bfloat16((hv[b] - df32(__bfloat162float(hi), 0.f)).hi);
          }
          if (HAh) {
            const __half hi = __float2half(hv[b].hi);
            HAh[e] = hi;
            if (split_lo) HAh[m * N + e] = __float2half((hv[b] - df32(__half2float(hi), 0.f)).hi);
          }
        }
      }
    }
  }
  if (hamax) {
    // non-negative floats order as their bit patterns
    const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(hmax));
    if (lane == 0 && mb > 0u) atomicMax(hamax, mb);
  }
}

// Rows [i_begin, i_end) of the innovation step: FP64 arithmetic for FP64 ensembles,
// double-float for FP32 ones.
template <typename VT>
__device__ __forceinline__ void innov_rows(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ HA64, float* __restrict__ HA32, double* __restrict__ D,
    float* __restrict__ B32, __nv_bfloat16* __restrict__ HAb, __half* __restrict__ HAh,
    int split_lo, df32* __restrict__ HAdf, df32* __restrict__ Ddf, int64_t i_begin, int64_t i_end,
    int64_t warp, int64_t nwarps, unsigned* hamax = nullptr) {
  if constexpr (sizeof(VT) == 4)
    innov_rows_df<VT>(Xf, rowptr, col, w, y, r, E, emode, seed, counter, m, N, HA64, HA32, D, B32,
                      HAb, HAh, split_lo, HAdf, Ddf, i_begin, i_end, warp, nwarps, hamax);
  else
    innov_rows_f64<VT>(Xf, rowptr, col, w, y, r, E, emode, seed, counter, m, N, HA64, HA32, D, B32,
                       HAb, HAh, split_lo, HAdf, Ddf, i_begin, i_end, warp, nwarps);
}

}  // namespace enkf
