// Device building blocks of the persistent CG solvers (shared by kernels_fp.cu and
// kernels_tc.cu): tiling constants, 4-wide fragments, fixed-order reductions, the two
// contraction passes of the matvec (Eq. matvec_decomp) and the fused CG step.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace enkf {

// ------------------------------------------------------------------ tiling
// NT = padded column count (N <= NT). Pass A (T = HA^T V): MA x MA register tile per
// thread over (k, j), TRA rows of HA and V staged in shared memory per step, RG row groups.
// Pass B (Q = HA T): 4 x 4 register tile per thread over (i, j), TRB rows per tile.
// Phase timer slots of the persistent solves (CTA 0, thread 0): accumulated ns per phase.
enum : int { PH_SETUP = 0, PH_PASS, PH_BAR1, PH_RED, PH_BAR2, PH_SCAL, PH_REFRESH, PH_COUNT = 8 };

template <int NT> struct Tile;
template <> struct Tile<32> { static constexpr int MA = 4, TRA = 32, TRB = 128; };
template <> struct Tile<64> { static constexpr int MA = 4, TRA = 32, TRB = 64; };
template <> struct Tile<128> { static constexpr int MA = 8, TRA = 16, TRB = 32; };

// Fused CG pass tile: TR rows of HA, r, p, s, x staged per step; MR rows per thread in the
// update (pass-B mapping, NT/4 column groups of 4).
template <typename CT, int NT> struct FTile;
template <int NT> struct FTile<float, NT> { static constexpr int MR = 4, TR = (1024 / NT) * 4; };
template <> struct FTile<double, 32> { static constexpr int MR = 2, TR = 64; };
template <> struct FTile<double, 64> { static constexpr int MR = 2, TR = 32; };
template <> struct FTile<double, 128> { static constexpr int MR = 1, TR = 8; };

// shared scalars: 12 FP64 arrays, 4 int arrays, 2 VT-sized (<= 8 B) arrays, each of length NT
template <int NT> __host__ __device__ constexpr int scalar_bytes() { return NT * 8 * 12 + NT * 4 * 4 + NT * 8 * 2; }
template <int NT> __host__ __device__ constexpr int refresh_union_bytes() {
  constexpr int MA = Tile<NT>::MA, TRA = Tile<NT>::TRA, TRB = Tile<NT>::TRB;
  constexpr int NG = NT / MA, RG = kThreads / (NG * NG);
  constexpr int a = 2 * TRA * NT * 8 + TRA * 8;
  constexpr int a2 = RG * NT * NT * 8;
  constexpr int a3 = 2 * RG * NG * NT * 8;
  constexpr int b = NT * (NT + 2) * 8 + TRB * (NT + 2) * 8;
  constexpr int m1 = a > a2 ? a : a2;
  constexpr int m2 = m1 > a3 ? m1 : a3;
  return m2 > b ? m2 : b;
}
template <typename CT, int NT> __host__ __device__ constexpr int passF_bytes() {
  constexpr int LD = NT + 16 / (int)sizeof(CT), TR = FTile<CT, NT>::TR;
  return NT * LD * (int)sizeof(CT) + 5 * TR * LD * (int)sizeof(CT) + TR * (int)sizeof(CT);
}
// FP32 solves use the double-buffered fused pass (passF_async)
template <typename VT, int NT> __host__ __device__ constexpr bool async_passF() {
  return sizeof(VT) == 4;
}
// NT = 128: x is read into registers instead of staged, so that two tiles fit in shared memory
template <int NT> __host__ __device__ constexpr bool async_xreg() { return NT == 128; }
template <int NT> __host__ __device__ constexpr int passF_async_bytes();
template <int NT> struct DFTile;
template <int NT> __host__ __device__ constexpr int passH_async_bytes();
template <typename VT, int NT> __host__ __device__ constexpr int union_bytes() {
  constexpr int f0 = async_passF<VT, NT>() ? passF_async_bytes<NT>() : passF_bytes<VT, NT>();
  constexpr int f = sizeof(VT) == 4 && passH_async_bytes<NT>() > f0 ? passH_async_bytes<NT>() : f0;
  constexpr int d = sizeof(VT) == 4 ? DFTile<NT>::bytes : 0;   // pipelined double-float refresh
  constexpr int m1 = refresh_union_bytes<NT>() > f ? refresh_union_bytes<NT>() : f;
  return m1 > d ? m1 : d;
}
template <typename VT, int NT> __host__ __device__ constexpr int solve_smem_bytes() {
  return scalar_bytes<NT>() + kThreads * 8 + union_bytes<VT, NT>();
}

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }


// ------------------------------------------------------------------ double-float arithmetic
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2 (about 44
// significant bits). Products and sums use the error-free transformations of Dekker and
// Knuth (TwoProd through FMA, TwoSum, Fast2Sum), written with the _rn intrinsics so that the
// compiler cannot contract or reorder them. On this GPU FP32 issues at 64x the FP64 rate, so
// a double-float multiply-add (15 FP32 instructions) is about 4x faster than a native DFMA.
struct __align__(8) df32 {
  float hi, lo;
  __host__ __device__ df32() : hi(0.f), lo(0.f) {}
  __device__ explicit df32(double x) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
  }
  __device__ df32(float h, float l) : hi(h), lo(l) {}
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ df32 df_fast2sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df32(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// c + a b
__device__ __forceinline__ df32 fma(const df32& a, const df32& b, const df32& c) {
  const float ph = __fmul_rn(a.hi, b.hi);
  float pl = __fmaf_rn(a.hi, b.hi, -ph);
  pl = __fmaf_rn(a.hi, b.lo, pl);
  pl = __fmaf_rn(a.lo, b.hi, pl);
  float s, e;
  df_two_sum(c.hi, ph, s, e);
  e = __fadd_rn(e, __fadd_rn(c.lo, pl));
  return df_fast2sum(s, e);
}
// keep the FP32 / FP64 fma overloads visible next to the double-float one
using ::fma;

__device__ __forceinline__ df32 operator+(const df32& a, const df32& b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_fast2sum(s, e);
}
__device__ __forceinline__ df32 operator-(const df32& a) { return df32(-a.hi, -a.lo); }
__device__ __forceinline__ df32 operator-(const df32& a, const df32& b) { return a + (-b); }
__device__ __forceinline__ df32 operator*(const df32& a, const df32& b) {
  const float ph = __fmul_rn(a.hi, b.hi);
  float pl = __fmaf_rn(a.hi, b.hi, -ph);
  pl = __fmaf_rn(a.hi, b.lo, pl);
  pl = __fmaf_rn(a.lo, b.hi, pl);
  return df_fast2sum(ph, pl);
}
__device__ __forceinline__ df32& operator+=(df32& a, const df32& b) { a = a + b; return a; }

// A running sum of double-float products kept as an unnormalised pair (s, c): each product's
// high part enters s through TwoSum, and its rounding error, the cross terms of the operands'
// low parts and the TwoSum error are added to c. renorm() folds c back into s and is called
// every few terms, so c stays within a few ulp(s) (the compensated dot product of Ogita,
// Rump and Oishi, renormalised in short blocks): 12 FP32 operations per term instead of the
// 15 of a renormalising double-float multiply-add, with the same double-float accuracy.
struct DFAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(const df32& a, const df32& b) {
    const float ph = __fmul_rn(a.hi, b.hi);
    float pl = __fmaf_rn(a.hi, b.hi, -ph);
    pl = __fmaf_rn(a.hi, b.lo, pl);
    pl = __fmaf_rn(a.lo, b.hi, pl);
    float t, e;
    df_two_sum(s, ph, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pl));
  }
  __device__ __forceinline__ void renorm() {
    const df32 v = df_fast2sum(s, c);
    s = v.hi;
    c = v.lo;
  }
  __device__ __forceinline__ df32 value() const { return df_fast2sum(s, c); }
};

// ------------------------------------------------------------------ 4-wide fragments
template <typename CT> __device__ __forceinline__ void load_vec(CT* d, const CT* s, int n);
template <> __device__ __forceinline__ void load_vec<float>(float* d, const float* s, int n) {
  for (int q = 0; q < n; q += 4) {
    const float4 v = *reinterpret_cast<const float4*>(s + q);
    d[q] = v.x; d[q + 1] = v.y; d[q + 2] = v.z; d[q + 3] = v.w;
  }
}
template <> __device__ __forceinline__ void load_vec<double>(double* d, const double* s, int n) {
  for (int q = 0; q < n; q += 2) {
    const double2 v = *reinterpret_cast<const double2*>(s + q);
    d[q] = v.x; d[q + 1] = v.y;
  }
}
template <> __device__ __forceinline__ void load_vec<df32>(df32* d, const df32* s, int n) {
  for (int q = 0; q < n; q += 2) {
    const float4 v = *reinterpret_cast<const float4*>(s + q);
    d[q] = df32(v.x, v.y);
    d[q + 1] = df32(v.z, v.w);
  }
}
template <typename CT> __device__ __forceinline__ void store_vec4(CT* d, const CT* s);
template <> __device__ __forceinline__ void store_vec4<float>(float* d, const float* s) {
  *reinterpret_cast<float4*>(d) = make_float4(s[0], s[1], s[2], s[3]);
}
template <> __device__ __forceinline__ void store_vec4<double>(double* d, const double* s) {
  *reinterpret_cast<double2*>(d) = make_double2(s[0], s[1]);
  *reinterpret_cast<double2*>(d + 2) = make_double2(s[2], s[3]);
}
template <> __device__ __forceinline__ void store_vec4<df32>(df32* d, const df32* s) {
  *reinterpret_cast<float4*>(d) = make_float4(s[0].hi, s[0].lo, s[1].hi, s[1].lo);
  *reinterpret_cast<float4*>(d + 2) = make_float4(s[2].hi, s[2].lo, s[3].hi, s[3].lo);
}
// row pointer p, columns j0..j0+3 (vec: N % 4 == 0, so the 4 columns exist and are aligned)
template <typename CT>
__device__ __forceinline__ void ld4(CT (&d)[4], const CT* p, int j0, int N, bool vec) {
  if (vec) { load_vec<CT>(d, p + j0, 4); return; }
#pragma unroll
  for (int y = 0; y < 4; ++y) d[y] = (j0 + y < N) ? p[j0 + y] : CT(0);
}
template <typename CT>
__device__ __forceinline__ void st4(CT* p, int j0, int N, bool vec, const CT (&s)[4]) {
  if (vec) { store_vec4<CT>(p + j0, s); return; }
#pragma unroll
  for (int y = 0; y < 4; ++y)
    if (j0 + y < N) p[j0 + y] = s[y];
}

// ------------------------------------------------------------------ reductions
// Block partial of a per-column sum over the CTA's rows: f(i, j, acc) is called once per
// element (i in [row0,row1), j < N); the per-column totals land in out[0..NT).
template <int NT, class F>
__device__ __forceinline__ void rows_reduce(int64_t row0, int64_t row1, int N, F f, double* out,
                                            double* scratch) {
  constexpr int L = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, lane = t / NT;
  double acc = 0.0;
  if (j < N)
    for (int64_t i = row0 + lane; i < row1; i += L) f(i, j, acc);
  scratch[t] = acc;
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < L; ++q) s += scratch[q * NT + t];
    out[t] = s;
  }
  __syncthreads();
}

// Every CTA sums the G block partials part[b*NT + j] (b < G, j < N) in the same fixed order,
// so all CTAs obtain bitwise identical totals (and take identical decisions).
template <int NT>
__device__ __forceinline__ void reduce_all(const double* __restrict__ part, int G, int N,
                                           double* out, double* scratch) {
  constexpr int Q = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, q = t / NT;
  double s = 0.0;
  if (j < N) {
    const int b0 = (int)((int64_t)q * G / Q), b1 = (int)((int64_t)(q + 1) * G / Q);
#pragma unroll 8
    for (int b = b0; b < b1; ++b) s += __ldcg(part + (int64_t)b * NT + j);
  }
  scratch[t] = s;
  __syncthreads();
  if (t < NT) {
    double v = 0.0;
    for (int qq = 0; qq < Q; ++qq) v += scratch[qq * NT + t];
    out[t] = v;
  }
  __syncthreads();
}

// CTA b (of G) sums its slice of the NE-long partial vectors part[g*NE + e] over g < G (fixed
// order) and writes red[e]. Entries e < n_f32 are written in FP32 instead, at
// reinterpret_cast<float*>(red)[e] (bytes [0, 4 n_f32), so they never overlap an FP64 entry
// e >= n_f32): the CG steps of the FP32 and tensor-core modes read T only as FP32, and one
// conversion per entry here replaces N^2 FP64 conversions in every CTA.
__device__ __forceinline__ void store_reduced(double* __restrict__ red, int e, int n_f32, double v) {
  if (e < n_f32) reinterpret_cast<float*>(red)[e] = (float)v;
  else red[e] = v;
}

__device__ __forceinline__ void reduce_slice(const double* __restrict__ part, int G, int NE,
                                             double* __restrict__ red, double* scratch,
                                             int b, int n_f32 = 0) {
  const int t = threadIdx.x;
  const int chunk = (NE + G - 1) / G;
  const int e0 = b * chunk;
  const int cnt = min(NE, e0 + chunk) - e0;
  if (cnt <= 0) return;
  if (cnt >= kThreads) {
    for (int e = e0 + t; e < e0 + cnt; e += kThreads) {
      double s = 0.0;
#pragma unroll 8
      for (int g = 0; g < G; ++g) s += __ldcg(part + (int64_t)g * NE + e);
      store_reduced(red, e, n_f32, s);
    }
    return;
  }
  const int parts = kThreads / cnt;
  const int q = t / cnt, el = t % cnt;
  double s = 0.0;
  if (q < parts) {
    const int g0 = (int)((int64_t)q * G / parts), g1 = (int)((int64_t)(q + 1) * G / parts);
#pragma unroll 8
    for (int g = g0; g < g1; ++g) s += __ldcg(part + (int64_t)g * NE + e0 + el);
  }
  scratch[t] = s;
  __syncthreads();
  if (t < cnt) {
    double v = 0.0;
    for (int qq = 0; qq < parts; ++qq) v += scratch[qq * cnt + t];
    store_reduced(red, e0 + t, n_f32, v);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ pass A
// out[k*N + j] = sum_i HA[i][k] V[i][j] over the CTA's rows and (want_s)
// out[N*N + j] = sum_i r_i V[i][j]^2 and out[N*N + N + j] = sum_i V[i][j]^2, where
// pro(i, j0, v) produces (and may store) the four values V[i][j0..j0+3]. Per-thread partial
// sums are kept in CT.
template <typename CT, int NT, class Pro, bool PC = false>
__device__ __forceinline__ void passA(const CT* __restrict__ HA, int64_t row0, int64_t row1,
                                      int N, const CT* __restrict__ rv, bool want_s, Pro& pro,
                                      unsigned char* uni, double* __restrict__ out) {
  constexpr int MA = Tile<NT>::MA, TRA = Tile<NT>::TRA;
  constexpr int NG = NT / MA, TPG = NG * NG, RG = kThreads / TPG, C4 = NT / 4;
  CT* sA = reinterpret_cast<CT*>(uni);
  CT* sV = sA + TRA * NT;
  CT* sR = sV + TRA * NT;
  const int t = threadIdx.x, g = t / TPG, u = t % TPG, tj = u % NG, tk = u / NG;
  const int k0 = tk * MA, j0 = tj * MA;
  const bool vec = (N & 3) == 0;
  CT acc[MA][MA];
#pragma unroll
  for (int x = 0; x < MA; ++x)
#pragma unroll
    for (int y = 0; y < MA; ++y) acc[x][y] = CT(0);
  CT sacc[MA], gacc[MA];
#pragma unroll
  for (int y = 0; y < MA; ++y) { sacc[y] = CT(0); gacc[y] = CT(0); }

  for (int64_t i0 = row0; i0 < row1; i0 += TRA) {
    __syncthreads();
#pragma unroll
    for (int c = t; c < TRA * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      CT a[4] = {CT(0), CT(0), CT(0), CT(0)}, v[4] = {CT(0), CT(0), CT(0), CT(0)};
      if (i < row1 && c0 < N) {
        ld4<CT>(a, HA + i * N, c0, N, vec);
        pro(i, c0, v, vec);
      }
      store_vec4<CT>(sA + ii * NT + c0, a);
      store_vec4<CT>(sV + ii * NT + c0, v);
    }
    if (t < TRA) {
      const int64_t i = i0 + t;
      sR[t] = (want_s && i < row1) ? rv[i] : CT(0);
    }
    __syncthreads();
    const int nrows = (int)imin64(TRA, row1 - i0);
    for (int ii = g; ii < nrows; ii += RG) {
      CT a[MA], v[MA];
      load_vec<CT>(a, sA + ii * NT + k0, MA);
      load_vec<CT>(v, sV + ii * NT + j0, MA);
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) acc[x][y] = fma(a[x], v[y], acc[x][y]);
      if (((ii / RG) % NG) == tk) {
        const CT ri = sR[ii];
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          sacc[y] = fma(ri * v[y], v[y], sacc[y]);
          const CT gv = PC ? ri * v[y] : v[y];   // preconditioned: v = b / r, so r v = b
          gacc[y] = fma(gv, gv, gacc[y]);
        }
      }
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(uni);
  if (RG > 1) {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) red[(g * NT + k0 + x) * NT + j0 + y] = (double)acc[x][y];
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          const int k = k0 + x, j = j0 + y;
          double s = 0.0;
          for (int gg = 0; gg < RG; ++gg) s += red[(gg * NT + k) * NT + j];
          if (k < N && j < N) out[k * N + j] = s;
        }
    }
  } else {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) {
        const int k = k0 + x, j = j0 + y;
        if (k < N && j < N) out[k * N + j] = (double)acc[x][y];
      }
  }
  __syncthreads();
#pragma unroll
  for (int y = 0; y < MA; ++y) {
    red[(g * NG + tk) * NT + j0 + y] = (double)sacc[y];
    red[RG * NG * NT + (g * NG + tk) * NT + j0 + y] = (double)gacc[y];
  }
  __syncthreads();
  if (t < N) {
    double s = 0.0, q2 = 0.0;
    for (int q = 0; q < RG * NG; ++q) {
      s += red[q * NT + t];
      q2 += red[RG * NG * NT + q * NT + t];
    }
    out[N * N + t] = want_s ? s : 0.0;
    out[N * N + N + t] = q2;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ pass B
// For each of the CTA's rows i and 4-column fragment j0: acc[y] = sum_k HA[i][k] T[k][j0+y];
// epi.prefetch loads the fragment's operands before the contraction, epi.apply updates the
// fragment and accumulates squared residuals into rr[y] (CT). rr_out[j] = block sum (FP64).
template <typename CT, int NT, class Epi>
__device__ __forceinline__ void passB(const CT* __restrict__ HA, int64_t row0, int64_t row1,
                                      int N, const CT* sT, unsigned char* sHbytes, Epi& epi,
                                      double* rr_out) {
  constexpr int PB = 16 / (int)sizeof(CT), LD = NT + PB, TRB = Tile<NT>::TRB, C4 = NT / 4;
  constexpr int NJ = NT / 4, NI = kThreads / NJ;
  static_assert(NI * 4 == TRB, "tile");
  CT* sH = reinterpret_cast<CT*>(sHbytes);
  const int t = threadIdx.x, tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * 4;
  const bool vec = (N & 3) == 0;
  CT rr[4] = {CT(0), CT(0), CT(0), CT(0)};
  for (int64_t i0 = row0; i0 < row1; i0 += TRB) {
    __syncthreads();
#pragma unroll
    for (int c = t; c < TRB * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      CT a[4] = {CT(0), CT(0), CT(0), CT(0)};
      if (i < row1 && c0 < N) ld4<CT>(a, HA + i * N, c0, N, vec);
#pragma unroll
      for (int y = 0; y < 4; ++y) sH[ii * LD + c0 + y] = a[y];
    }
    // FP32 fragments are loaded before the contraction (latency overlap); FP64 passes are
    // DFMA-bound, so their fragments are loaded just before use to save registers
    constexpr int NF = Epi::kPrefetch ? 4 : 1;
    typename Epi::Frag frag[NF];
    if constexpr (Epi::kPrefetch) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int64_t i = i0 + r0 + x;
        if (i < row1 && j0 < N) epi.prefetch(i, j0, frag[x], vec);
      }
    }
    __syncthreads();
    CT acc[4][4];
    if constexpr (std::is_same<CT, df32>::value) {
      // double-float: the products enter unnormalised (sum, error) pairs, renormalised every
      // 4 terms (DFAcc), as in refreshB_async
      DFAcc dacc[4][4];
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        df32 a[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = sH[(r0 + x) * LD + k];
        load_vec<df32>(bv, sT + k * LD + j0, 4);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) dacc[x][y].add(a[x], bv[y]);
        if ((k & 3) == 3) {
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) dacc[x][y].renorm();
        }
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = dacc[x][y].value();
    } else {
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = CT(0);
    if (N == NT) {
#pragma unroll 8
      for (int k = 0; k < NT; ++k) {
        CT a[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = sH[(r0 + x) * LD + k];
        load_vec<CT>(bv, sT + k * LD + j0, 4);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bv[y], acc[x][y]);
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        CT a[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = sH[(r0 + x) * LD + k];
        load_vec<CT>(bv, sT + k * LD + j0, 4);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bv[y], acc[x][y]);
      }
    }
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int64_t i = i0 + r0 + x;
      if (i < row1 && j0 < N) {
        if constexpr (Epi::kPrefetch) {
          epi.apply(i, j0, acc[x], frag[x], rr, vec);
        } else {
          epi.prefetch(i, j0, frag[0], vec);
          epi.apply(i, j0, acc[x], frag[0], rr, vec);
        }
      }
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(sHbytes);
#pragma unroll
  for (int y = 0; y < 4; ++y) red[ti * NT + j0 + y] = (double)rr[y];
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < NI; ++q) s += red[q * NT + t];
    rr_out[t] = s;
  }
  __syncthreads();
}

// Stage the reduced N x N matrix (FP64 in global) into shared memory as CT with stride
// NT + 16/sizeof(CT), zero-padded to NT x NT.
template <typename CT, int NT>
__device__ __forceinline__ void stage_T(const double* __restrict__ Tred, int N, CT* sT) {
  constexpr int LD = NT + 16 / (int)sizeof(CT);
  for (int e = threadIdx.x; e < NT * LD; e += kThreads) {
    const int k = e / LD, j = e % LD;
    sT[e] = (k < N && j < N) ? (CT)__ldcg(Tred + k * N + j) : CT(0);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ fused CG pass
// Chronopoulos-Gear form of CG (algebraically the Hestenes-Stiefel recurrences): with
// s = S p carried along, u = S r, gamma = (r, r) and delta = (r, S r) =
// ||HA^T r||^2/(N-1) + sum_i r_i r_i^2, a step needs only one reduction:
//   beta = gamma/gamma_old, alpha = gamma / (delta - beta gamma/alpha_old),
//   p = r + beta p, s = u + beta s, x += alpha p, r -= alpha s.
// One pass over the CTA's rows does the step and, on the same shared-memory tile, the
// partial HA^T r_new, sum r_i r_new^2 and sum r_new^2 of the next step: out = [T | sig | gam].
//
// With the Jacobi preconditioner M = R (PC), the step is the preconditioned form with
// z = R^{-1} r: w = S z = HA (HA^T z)/(N-1) + r, gamma = (r, z), delta = (z, S z) =
// ||HA^T z||^2/(N-1) + gamma, p = z + beta p, s = w + beta s, and the next partials are
// [HA^T z_new | (r_new, z_new) | (r_new, r_new)].
template <typename CT, int NT, bool PC = false>
__device__ __forceinline__ void passF(const CT* __restrict__ HA, int64_t row0, int64_t row1, int N,
                                      CT* X, CT* Res, CT* P, CT* Sv, const CT* __restrict__ rv,
                                      const CT* sT, const CT* alpha, const CT* beta, CT vinv,
                                      unsigned char* tiles, double* __restrict__ out) {
  constexpr int LD = NT + 16 / (int)sizeof(CT);
  constexpr int MR = FTile<CT, NT>::MR, TR = FTile<CT, NT>::TR, C4 = NT / 4;
  constexpr int NJ = NT / 4, NI = kThreads / NJ;
  static_assert(NI * MR == TR, "fused tile");
  constexpr int MA = Tile<NT>::MA, NG = NT / MA, TPG = NG * NG, RG = kThreads / TPG;
  CT* sH = reinterpret_cast<CT*>(tiles);
  CT* sR = sH + TR * LD;
  CT* sP = sR + TR * LD;
  CT* sS = sP + TR * LD;
  CT* sX = sS + TR * LD;
  CT* sRv = sX + TR * LD;
  const int t = threadIdx.x;
  const int tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * MR;                  // update map
  const int g = t / TPG, u = t % TPG, gj = u % NG, gk = u / NG, k0 = gk * MA, ja = gj * MA;  // Gram map
  const bool vec = (N & 3) == 0;
  CT accT[MA][MA];
#pragma unroll
  for (int x = 0; x < MA; ++x)
#pragma unroll
    for (int y = 0; y < MA; ++y) accT[x][y] = CT(0);
  CT sig[4] = {CT(0), CT(0), CT(0), CT(0)}, gam[4] = {CT(0), CT(0), CT(0), CT(0)};
  CT al[4], be[4];
#pragma unroll
  for (int y = 0; y < 4; ++y) { al[y] = alpha[j0 + y]; be[y] = beta[j0 + y]; }

  for (int64_t i0 = row0; i0 < row1; i0 += TR) {
    __syncthreads();
#pragma unroll
    for (int c = t; c < TR * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      CT a[4] = {CT(0), CT(0), CT(0), CT(0)}, rr[4] = {CT(0), CT(0), CT(0), CT(0)};
      CT pp[4] = {CT(0), CT(0), CT(0), CT(0)}, ss[4] = {CT(0), CT(0), CT(0), CT(0)};
      CT xx[4] = {CT(0), CT(0), CT(0), CT(0)};
      if (i < row1 && c0 < N) {
        ld4<CT>(a, HA + i * N, c0, N, vec);
        ld4<CT>(rr, Res + i * N, c0, N, vec);
        ld4<CT>(pp, P + i * N, c0, N, vec);
        ld4<CT>(ss, Sv + i * N, c0, N, vec);
        ld4<CT>(xx, X + i * N, c0, N, vec);
      }
      store_vec4<CT>(sH + ii * LD + c0, a);
      store_vec4<CT>(sR + ii * LD + c0, rr);
      store_vec4<CT>(sP + ii * LD + c0, pp);
      store_vec4<CT>(sS + ii * LD + c0, ss);
      store_vec4<CT>(sX + ii * LD + c0, xx);
    }
    if (t < TR) {
      const int64_t i = i0 + t;
      sRv[t] = i < row1 ? rv[i] : CT(0);
    }
    __syncthreads();
    // u = HA T / (N-1) + r_i r
    CT acc[MR][4];
#pragma unroll
    for (int x = 0; x < MR; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = CT(0);
    if (N == NT) {
#pragma unroll 8
      for (int k = 0; k < NT; ++k) {
        CT a[MR], bv[4];
#pragma unroll
        for (int x = 0; x < MR; ++x) a[x] = sH[(r0 + x) * LD + k];
        load_vec<CT>(bv, sT + k * LD + j0, 4);
#pragma unroll
        for (int x = 0; x < MR; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bv[y], acc[x][y]);
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        CT a[MR], bv[4];
#pragma unroll
        for (int x = 0; x < MR; ++x) a[x] = sH[(r0 + x) * LD + k];
        load_vec<CT>(bv, sT + k * LD + j0, 4);
#pragma unroll
        for (int x = 0; x < MR; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], bv[y], acc[x][y]);
      }
    }
    // the CG step on the thread's MR x 4 fragment
#pragma unroll
    for (int x = 0; x < MR; ++x) {
      const int row = r0 + x;
      const int64_t i = i0 + row;
      if (i < row1 && j0 < N) {
        const CT ri = sRv[row];
        CT rv4[4], pv4[4], sv4[4], xv4[4], pn[4], sn[4], xn[4], rn[4];
        load_vec<CT>(rv4, sR + row * LD + j0, 4);
        load_vec<CT>(pv4, sP + row * LD + j0, 4);
        load_vec<CT>(sv4, sS + row * LD + j0, 4);
        load_vec<CT>(xv4, sX + row * LD + j0, 4);
        const CT rinv = PC ? CT(1) / ri : CT(0);
        CT zn[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          // plain: z = r, w = S r = HA T/(N-1) + R r; preconditioned: z = r / R, w = HA T/(N-1) + r
          const CT zz = PC ? rv4[y] * rinv : rv4[y];
          const CT ww = PC ? fma(acc[x][y], vinv, rv4[y]) : fma(acc[x][y], vinv, ri * rv4[y]);
          // beta == 0 (first step, frozen columns) selects p = z, s = w without reading the
          // old p, s (which may hold anything, including NaN bit patterns)
          pn[y] = be[y] == CT(0) ? zz : fma(be[y], pv4[y], zz);
          sn[y] = be[y] == CT(0) ? ww : fma(be[y], sv4[y], ww);
          xn[y] = fma(al[y], pn[y], xv4[y]);
          rn[y] = fma(-al[y], sn[y], rv4[y]);
          zn[y] = PC ? rn[y] * rinv : rn[y];
          sig[y] = PC ? fma(rn[y], zn[y], sig[y]) : fma(ri * rn[y], rn[y], sig[y]);
          gam[y] = fma(rn[y], rn[y], gam[y]);
        }
        st4<CT>(P + i * N, j0, N, vec, pn);
        st4<CT>(Sv + i * N, j0, N, vec, sn);
        st4<CT>(X + i * N, j0, N, vec, xn);
        st4<CT>(Res + i * N, j0, N, vec, rn);
        store_vec4<CT>(sR + row * LD + j0, zn);
      }
    }
    __syncthreads();
    // next step's partial Gram HA^T r_new on the same tile
    const int nrows = (int)imin64(TR, row1 - i0);
    for (int ii = g; ii < nrows; ii += RG) {
      CT a[MA], v[MA];
      load_vec<CT>(a, sH + ii * LD + k0, MA);
      load_vec<CT>(v, sR + ii * LD + ja, MA);
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) accT[x][y] = fma(a[x], v[y], accT[x][y]);
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(tiles);
  if (RG > 1) {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) red[(g * NT + k0 + x) * NT + ja + y] = (double)accT[x][y];
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          const int k = k0 + x, j = ja + y;
          double s = 0.0;
          for (int gg = 0; gg < RG; ++gg) s += red[(gg * NT + k) * NT + j];
          if (k < N && j < N) out[k * N + j] = s;
        }
    }
  } else {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) {
        const int k = k0 + x, j = ja + y;
        if (k < N && j < N) out[k * N + j] = (double)accT[x][y];
      }
  }
  __syncthreads();
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    red[ti * NT + j0 + y] = (double)sig[y];
    red[NI * NT + ti * NT + j0 + y] = (double)gam[y];
  }
  __syncthreads();
  if (t < N) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < NI; ++q) {
      a += red[q * NT + t];
      b += red[NI * NT + q * NT + t];
    }
    out[N * N + t] = a;
    out[N * N + N + t] = b;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ fused CG pass, pipelined
// The FP32 fused step of passF for NT <= 64 with the row tiles double-buffered: the next
// tile's HA, r, p, s, x and r_i are copied global -> shared with cp.async (16-byte pieces,
// zero-filled past the CTA's rows and past N) while the current tile is computed. Needs
// N % 4 == 0 (16-byte aligned rows). The u = HA T contraction reads HA four k at a time.
// Same arithmetic, partial sums and output as passF (fixed order).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

template <int NT> __host__ __device__ constexpr int passF_async_bytes() {
  constexpr int LD = NT + 4, TR = FTile<float, NT>::TR, NS = async_xreg<NT>() ? 4 : 5;
  return NT * LD * 4 + 2 * (NS * TR * LD + TR) * 4;
}

template <int NT, bool PC>
__device__ __forceinline__ void passF_async(const float* __restrict__ HA, int64_t row0, int64_t row1, int N,
                                            float* X, float* Res, float* P, float* Sv,
                                            const float* __restrict__ rv, const float* sT,
                                            const float* alpha, const float* beta, float vinv,
                                            unsigned char* tiles, double* __restrict__ out) {
  constexpr int LD = NT + 4;
  constexpr int MR = FTile<float, NT>::MR, TR = FTile<float, NT>::TR, C4 = NT / 4;
  constexpr int NJ = NT / 4, NI = kThreads / NJ;
  static_assert(NI * MR == TR, "fused tile");
  constexpr int MA = Tile<NT>::MA, NG = NT / MA, TPG = NG * NG, RG = kThreads / TPG;
  constexpr bool XREG = async_xreg<NT>();
  constexpr int NS = XREG ? 4 : 5;          // staged arrays: HA, r, p, S p (, x)
  constexpr int BUF = NS * TR * LD + TR;   // floats per buffer
  float* const buf0 = reinterpret_cast<float*>(tiles);
  const int t = threadIdx.x;
  const int tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * MR;
  const int g = t / TPG, u = t % TPG, gj = u % NG, gk = u / NG, k0 = gk * MA, ja = gj * MA;
  float accT[MA][MA];
#pragma unroll
  for (int x = 0; x < MA; ++x)
#pragma unroll
    for (int y = 0; y < MA; ++y) accT[x][y] = 0.f;
  float sig[4] = {0.f, 0.f, 0.f, 0.f}, gam[4] = {0.f, 0.f, 0.f, 0.f};
  float al[4], be[4];
#pragma unroll
  for (int y = 0; y < 4; ++y) { al[y] = alpha[j0 + y]; be[y] = beta[j0 + y]; }

  // copy tile starting at row i0 into buffer b
  auto issue = [&](int64_t i0, int b) {
    float* sb = buf0 + b * BUF;
#pragma unroll
    for (int c = t; c < TR * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      const bool ok = i < row1 && c0 < N;
      const int64_t off = ok ? i * N + c0 : row0 * N;
      cp_async16(sb + 0 * TR * LD + ii * LD + c0, HA + off, ok);
      cp_async16(sb + 1 * TR * LD + ii * LD + c0, Res + off, ok);
      cp_async16(sb + 2 * TR * LD + ii * LD + c0, P + off, ok);
      cp_async16(sb + 3 * TR * LD + ii * LD + c0, Sv + off, ok);
      if (!XREG) cp_async16(sb + 4 * TR * LD + ii * LD + c0, X + off, ok);
    }
    if (t < TR) {
      const int64_t i = i0 + t;
      cp_async4(sb + NS * TR * LD + t, rv + (i < row1 ? i : row0), i < row1);
    }
    cp_async_commit();
  };

  int b = 0;
  if (row0 < row1) issue(row0, 0);
  for (int64_t i0 = row0; i0 < row1; i0 += TR, b ^= 1) {
    const bool more = i0 + TR < row1;
    if (more) {
      issue(i0 + TR, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* sH = buf0 + b * BUF;
    float* sR = buf0 + b * BUF + TR * LD;
    const float* sP = sR + TR * LD;
    const float* sS = sP + TR * LD;
    const float* sX = sS + TR * LD;                      // (NS == 5 only)
    const float* sRv = sS + (NS - 3) * TR * LD;
    // NT = 128: the thread's x fragment straight from global, in flight during the contraction
    float xg[MR][4];
    if (XREG) {
#pragma unroll
      for (int x = 0; x < MR; ++x) {
        const int64_t i = i0 + r0 + x;
#pragma unroll
        for (int y = 0; y < 4; ++y) xg[x][y] = 0.f;
        if (i < row1 && j0 < N) {
          const float4 v = *reinterpret_cast<const float4*>(X + i * N + j0);
          xg[x][0] = v.x; xg[x][1] = v.y; xg[x][2] = v.z; xg[x][3] = v.w;
        }
      }
    }
    // u = HA T (the 1/(N-1) is applied below); four k per step from float4 rows of HA
    float acc[MR][4];
#pragma unroll
    for (int x = 0; x < MR; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int k = 0; k < NT; k += 4) {
      float4 a4[MR];
#pragma unroll
      for (int x = 0; x < MR; ++x) a4[x] = *reinterpret_cast<const float4*>(sH + (r0 + x) * LD + k);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 b4 = *reinterpret_cast<const float4*>(sT + (k + kk) * LD + j0);
#pragma unroll
        for (int x = 0; x < MR; ++x) {
          const float av = kk == 0 ? a4[x].x : kk == 1 ? a4[x].y : kk == 2 ? a4[x].z : a4[x].w;
          acc[x][0] = fmaf(av, b4.x, acc[x][0]);
          acc[x][1] = fmaf(av, b4.y, acc[x][1]);
          acc[x][2] = fmaf(av, b4.z, acc[x][2]);
          acc[x][3] = fmaf(av, b4.w, acc[x][3]);
        }
      }
    }
    // the CG step on the thread's MR x 4 fragment (as passF)
#pragma unroll
    for (int x = 0; x < MR; ++x) {
      const int row = r0 + x;
      const int64_t i = i0 + row;
      if (i < row1 && j0 < N) {
        const float ri = sRv[row];
        const float4 rv4 = *reinterpret_cast<const float4*>(sR + row * LD + j0);
        const float4 pv4 = *reinterpret_cast<const float4*>(sP + row * LD + j0);
        const float4 sv4 = *reinterpret_cast<const float4*>(sS + row * LD + j0);
        const float4 xv4 = XREG ? make_float4(xg[x][0], xg[x][1], xg[x][2], xg[x][3])
                                : *reinterpret_cast<const float4*>(sX + row * LD + j0);
        const float rvv[4] = {rv4.x, rv4.y, rv4.z, rv4.w}, pvv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
        const float svv[4] = {sv4.x, sv4.y, sv4.z, sv4.w}, xvv[4] = {xv4.x, xv4.y, xv4.z, xv4.w};
        const float rinv = PC ? 1.f / ri : 0.f;
        float pn[4], sn[4], xn[4], rn[4], zn[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const float zz = PC ? rvv[y] * rinv : rvv[y];
          const float ww = PC ? fmaf(acc[x][y], vinv, rvv[y]) : fmaf(acc[x][y], vinv, ri * rvv[y]);
          pn[y] = be[y] == 0.f ? zz : fmaf(be[y], pvv[y], zz);
          sn[y] = be[y] == 0.f ? ww : fmaf(be[y], svv[y], ww);
          xn[y] = fmaf(al[y], pn[y], xvv[y]);
          rn[y] = fmaf(-al[y], sn[y], rvv[y]);
          zn[y] = PC ? rn[y] * rinv : rn[y];
          sig[y] = PC ? fmaf(rn[y], zn[y], sig[y]) : fmaf(ri * rn[y], rn[y], sig[y]);
          gam[y] = fmaf(rn[y], rn[y], gam[y]);
        }
        *reinterpret_cast<float4*>(P + i * N + j0) = make_float4(pn[0], pn[1], pn[2], pn[3]);
        *reinterpret_cast<float4*>(Sv + i * N + j0) = make_float4(sn[0], sn[1], sn[2], sn[3]);
        *reinterpret_cast<float4*>(X + i * N + j0) = make_float4(xn[0], xn[1], xn[2], xn[3]);
        *reinterpret_cast<float4*>(Res + i * N + j0) = make_float4(rn[0], rn[1], rn[2], rn[3]);
        *reinterpret_cast<float4*>(sR + row * LD + j0) = make_float4(zn[0], zn[1], zn[2], zn[3]);
      }
    }
    __syncthreads();
    // next step's partial Gram HA^T z_new on the same tile (rows past row1 are zero)
    const int nrows = (int)imin64(TR, row1 - i0);
    for (int ii = g; ii < nrows; ii += RG) {
      float a[MA], v[MA];
      load_vec<float>(a, sH + ii * LD + k0, MA);
      load_vec<float>(v, sR + ii * LD + ja, MA);
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) accT[x][y] = fmaf(a[x], v[y], accT[x][y]);
    }
    __syncthreads();   // this buffer is refilled by the copy issued in the next iteration
  }
  double* red = reinterpret_cast<double*>(tiles);
  if (RG > 1) {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) red[(g * NT + k0 + x) * NT + ja + y] = (double)accT[x][y];
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          const int k = k0 + x, j = ja + y;
          double s = 0.0;
          for (int gg = 0; gg < RG; ++gg) s += red[(gg * NT + k) * NT + j];
          if (k < N && j < N) out[k * N + j] = s;
        }
    }
  } else {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) {
        const int k = k0 + x, j = ja + y;
        if (k < N && j < N) out[k * N + j] = (double)accT[x][y];
      }
  }
  __syncthreads();
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    red[ti * NT + j0 + y] = (double)sig[y];
    red[NI * NT + ti * NT + j0 + y] = (double)gam[y];
  }
  __syncthreads();
  if (t < N) {
    double a = 0.0, bb = 0.0;
    for (int q = 0; q < NI; ++q) {
      a += red[q * NT + t];
      bb += red[NI * NT + q * NT + t];
    }
    out[N * N + t] = a;
    out[N * N + N + t] = bb;
  }
  __syncthreads();
}

// ------------------------------------------------------------------ one-reduction Hestenes-Stiefel step
// The FP32 inner solves use the textbook (Hestenes-Stiefel) recurrences with the matvec
// q = S p = HA T/(N-1) + R p formed from T = HA^T p in every step, arranged so that a step
// needs one pass over the rows and one grid reduction. T is carried in N x N space: with
// p_{k+1} = z_{k+1} + beta_k p_k, HA^T p_{k+1} = HA^T z_{k+1} + beta_k T_k, and
//   sum_i r_i p_{k+1,i}^2 = sum r_i z^2 + 2 beta_k sum r_i z p_k + beta_k^2 sum r_i p_k^2,
// so (p, S p) = ||T||^2/(N-1) + sum r_i p^2 comes from column sums of the pass. Pass k, with
// T_k staged, alpha_k and beta_{k-1}, per row: z_k = M^{-1} r_k (M = R preconditioned, else I),
// p_k = z_k + beta_{k-1} p_{k-1}, q_k = HA T_k/(N-1) + r_i p_k, x += alpha_k p_k,
// r -= alpha_k q_k, z_{k+1} = M^{-1} r_{k+1}; out = [HA^T z_{k+1} | (r, z) | (r, r) |
// sum r_i z^2 | sum r_i z p_k] (N^2 + 4N); with atomic_out the Gram is added into the FP32
// total at reinterpret_cast<float*>(out)[k*N + j] and the column sums into the FP64 totals
// (the layout reduce_slice leaves). In FP32 the Chronopoulos-Gear arrangement (one
// reduction, with S p carried by its own recurrence) needed about 1.7x the steps of this form on
// the 512^2 / N = 64 workload (67 against 40), and this form moves no S p vector.
template <int NT> __host__ __device__ constexpr int passH_async_bytes() {
  constexpr int LD = NT + 4, TR = FTile<float, NT>::TR, NS = async_xreg<NT>() ? 3 : 4;
  return NT * LD * 4 + 2 * (NS * TR * LD + TR) * 4;
}

template <int NT, bool PC, bool ASYNC>
__device__ __forceinline__ void passH(const float* __restrict__ HA, int64_t row0, int64_t row1, int N,
                                      float* X, float* Res, float* P, const float* __restrict__ rv,
                                      const float* sT, const float* alpha, const float* beta, float vinv,
                                      unsigned char* tiles, double* __restrict__ out, bool atomic_out = false) {
  constexpr int LD = NT + 4;
  constexpr int MR = FTile<float, NT>::MR, TR = FTile<float, NT>::TR, C4 = NT / 4;
  constexpr int NJ = NT / 4, NI = kThreads / NJ;
  static_assert(NI * MR == TR, "fused tile");
  constexpr int MA = Tile<NT>::MA, NG = NT / MA, TPG = NG * NG, RG = kThreads / TPG;
  constexpr bool XREG = async_xreg<NT>();
  constexpr int NS = XREG ? 3 : 4;          // staged arrays: HA, r, p (, x)
  constexpr int BUF = NS * TR * LD + TR;   // floats per buffer
  float* const buf0 = reinterpret_cast<float*>(tiles);
  const int t = threadIdx.x;
  const int tj = t % NJ, ti = t / NJ, j0 = tj * 4, r0 = ti * MR;
  const int g = t / TPG, u = t % TPG, gj = u % NG, gk = u / NG, k0 = gk * MA, ja = gj * MA;
  const bool vec = (N & 3) == 0;
  float accT[MA][MA];
#pragma unroll
  for (int x = 0; x < MA; ++x)
#pragma unroll
    for (int y = 0; y < MA; ++y) accT[x][y] = 0.f;
  float s1[4] = {0.f, 0.f, 0.f, 0.f}, s2[4] = {0.f, 0.f, 0.f, 0.f};
  float s3[4] = {0.f, 0.f, 0.f, 0.f}, s4[4] = {0.f, 0.f, 0.f, 0.f};
  float al[4], be[4];
#pragma unroll
  for (int y = 0; y < 4; ++y) { al[y] = alpha[j0 + y]; be[y] = beta[j0 + y]; }

  // copy the tile starting at row i0 into buffer b: 16-byte cp.async pieces (zero-filled past
  // the CTA's rows and past N) when rows are 16-byte aligned, else plain loads
  auto fill = [&](int64_t i0, int b) {
    float* sb = buf0 + b * BUF;
#pragma unroll
    for (int c = t; c < TR * C4; c += kThreads) {
      const int ii = c / C4, c0 = (c % C4) * 4;
      const int64_t i = i0 + ii;
      const bool ok = i < row1 && c0 < N;
      if (ASYNC) {
        const int64_t off = ok ? i * N + c0 : row0 * N;
        cp_async16(sb + 0 * TR * LD + ii * LD + c0, HA + off, ok);
        cp_async16(sb + 1 * TR * LD + ii * LD + c0, Res + off, ok);
        cp_async16(sb + 2 * TR * LD + ii * LD + c0, P + off, ok);
        if (!XREG) cp_async16(sb + 3 * TR * LD + ii * LD + c0, X + off, ok);
      } else {
        float a[4] = {0.f, 0.f, 0.f, 0.f}, rr[4] = {0.f, 0.f, 0.f, 0.f}, pp[4] = {0.f, 0.f, 0.f, 0.f};
        float xx[4] = {0.f, 0.f, 0.f, 0.f};
        if (ok) {
          ld4<float>(a, HA + i * N, c0, N, vec);
          ld4<float>(rr, Res + i * N, c0, N, vec);
          ld4<float>(pp, P + i * N, c0, N, vec);
          if (!XREG) ld4<float>(xx, X + i * N, c0, N, vec);
        }
        store_vec4<float>(sb + 0 * TR * LD + ii * LD + c0, a);
        store_vec4<float>(sb + 1 * TR * LD + ii * LD + c0, rr);
        store_vec4<float>(sb + 2 * TR * LD + ii * LD + c0, pp);
        if (!XREG) store_vec4<float>(sb + 3 * TR * LD + ii * LD + c0, xx);
      }
    }
    if (t < TR) {
      const int64_t i = i0 + t;
      if (ASYNC) cp_async4(sb + NS * TR * LD + t, rv + (i < row1 ? i : row0), i < row1);
      else sb[NS * TR * LD + t] = i < row1 ? rv[i] : 0.f;
    }
    if (ASYNC) cp_async_commit();
  };

  int b = 0;
  if (ASYNC && row0 < row1) fill(row0, 0);
  for (int64_t i0 = row0; i0 < row1; i0 += TR, b ^= ASYNC ? 1 : 0) {
    if (ASYNC) {
      if (i0 + TR < row1) {
        fill(i0 + TR, b ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else {
      fill(i0, 0);
    }
    __syncthreads();
    const float* sH = buf0 + b * BUF;
    float* sR = buf0 + b * BUF + TR * LD;
    const float* sP = sR + TR * LD;
    const float* sX = sP + TR * LD;                      // (NS == 4 only)
    const float* sRv = sR + (NS - 1) * TR * LD;
    // NT = 128: the thread's x fragment straight from global, in flight during the contraction
    float xg[MR][4];
    if (XREG) {
#pragma unroll
      for (int x = 0; x < MR; ++x) {
        const int64_t i = i0 + r0 + x;
#pragma unroll
        for (int y = 0; y < 4; ++y) xg[x][y] = 0.f;
        if (i < row1 && j0 < N) ld4<float>(xg[x], X + i * N, j0, N, vec);
      }
    }
    // u = HA T (the 1/(N-1) is applied below); four k per step from float4 rows of HA
    float acc[MR][4];
#pragma unroll
    for (int x = 0; x < MR; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll 4
    for (int k = 0; k < NT; k += 4) {
      float4 a4[MR];
#pragma unroll
      for (int x = 0; x < MR; ++x) a4[x] = *reinterpret_cast<const float4*>(sH + (r0 + x) * LD + k);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const float4 b4 = *reinterpret_cast<const float4*>(sT + (k + kk) * LD + j0);
#pragma unroll
        for (int x = 0; x < MR; ++x) {
          const float av = kk == 0 ? a4[x].x : kk == 1 ? a4[x].y : kk == 2 ? a4[x].z : a4[x].w;
          acc[x][0] = fmaf(av, b4.x, acc[x][0]);
          acc[x][1] = fmaf(av, b4.y, acc[x][1]);
          acc[x][2] = fmaf(av, b4.z, acc[x][2]);
          acc[x][3] = fmaf(av, b4.w, acc[x][3]);
        }
      }
    }
    // the step on the thread's MR x 4 fragment
#pragma unroll
    for (int x = 0; x < MR; ++x) {
      const int row = r0 + x;
      const int64_t i = i0 + row;
      if (i < row1 && j0 < N) {
        const float ri = sRv[row];
        const float4 rv4 = *reinterpret_cast<const float4*>(sR + row * LD + j0);
        const float4 pv4 = *reinterpret_cast<const float4*>(sP + row * LD + j0);
        const float4 xv4 = XREG ? make_float4(xg[x][0], xg[x][1], xg[x][2], xg[x][3])
                                : *reinterpret_cast<const float4*>(sX + row * LD + j0);
        const float rvv[4] = {rv4.x, rv4.y, rv4.z, rv4.w}, pvv[4] = {pv4.x, pv4.y, pv4.z, pv4.w};
        const float xvv[4] = {xv4.x, xv4.y, xv4.z, xv4.w};
        const float rinv = PC ? 1.f / ri : 0.f;
        float pn[4], xn[4], rn[4], zn[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const float zz = PC ? rvv[y] * rinv : rvv[y];
          // beta == 0 (first step, frozen columns) selects p = z without reading the old p
          pn[y] = be[y] == 0.f ? zz : fmaf(be[y], pvv[y], zz);
          const float q = fmaf(acc[x][y], vinv, ri * pn[y]);
          xn[y] = fmaf(al[y], pn[y], xvv[y]);
          rn[y] = fmaf(-al[y], q, rvv[y]);
          zn[y] = PC ? rn[y] * rinv : rn[y];
          s1[y] = fmaf(rn[y], zn[y], s1[y]);
          s2[y] = fmaf(rn[y], rn[y], s2[y]);
          s3[y] = fmaf(ri * zn[y], zn[y], s3[y]);
          s4[y] = fmaf(ri * zn[y], pn[y], s4[y]);
        }
        st4<float>(P + i * N, j0, N, vec, pn);
        st4<float>(X + i * N, j0, N, vec, xn);
        st4<float>(Res + i * N, j0, N, vec, rn);
        store_vec4<float>(sR + row * LD + j0, zn);
      }
    }
    __syncthreads();
    // next step's partial Gram HA^T z_new on the same tile; rows past row1 hold zeros in both
    // operands, so the loop runs over the whole tile (a fixed trip count the compiler unrolls
    // and pipelines)
#pragma unroll 8
    for (int ii = g; ii < TR; ii += RG) {
      float a[MA], v[MA];
      load_vec<float>(a, sH + ii * LD + k0, MA);
      load_vec<float>(v, sR + ii * LD + ja, MA);
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) accT[x][y] = fmaf(a[x], v[y], accT[x][y]);
    }
    __syncthreads();   // this buffer is refilled by the copy issued in the next iteration
  }
  double* red = reinterpret_cast<double*>(tiles);
  if (RG > 1) {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) red[(g * NT + k0 + x) * NT + ja + y] = (double)accT[x][y];
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          const int k = k0 + x, j = ja + y;
          double sum = 0.0;
          for (int gg = 0; gg < RG; ++gg) sum += red[(gg * NT + k) * NT + j];
          if (k < N && j < N) {
            if (atomic_out) atomicAdd(reinterpret_cast<float*>(out) + k * N + j, (float)sum);
            else out[k * N + j] = sum;
          }
        }
    }
  } else {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) {
        const int k = k0 + x, j = ja + y;
        if (k < N && j < N) {
          if (atomic_out) atomicAdd(reinterpret_cast<float*>(out) + k * N + j, accT[x][y]);
          else out[k * N + j] = (double)accT[x][y];
        }
      }
  }
  __syncthreads();
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    red[(0 * NI + ti) * NT + j0 + y] = (double)s1[y];
    red[(1 * NI + ti) * NT + j0 + y] = (double)s2[y];
    red[(2 * NI + ti) * NT + j0 + y] = (double)s3[y];
    red[(3 * NI + ti) * NT + j0 + y] = (double)s4[y];
  }
  __syncthreads();
  if (t < N) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double sum = 0.0;
      for (int q = 0; q < NI; ++q) sum += red[(c * NI + q) * NT + t];
      if (atomic_out) atomicAdd(out + N * N + c * N + t, sum);
      else out[N * N + c * N + t] = sum;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ double-float refresh, pipelined
// The two passes of the double-float refresh (N % 4 == 0) with the row tiles double-buffered
// through cp.async, as in passF_async: pass A at every NT, pass B for NT <= 64 (at NT = 128
// its staged T and two tiles do not fit, and passB runs synchronously with the same
// compensated pairs). Same partial sums as passA / passB with ProRefreshDF / EpiRefreshDF.
template <int NT> struct DFTile {
  static constexpr int MA = Tile<NT>::MA, NG = NT / MA, TPG = NG * NG, RG = kThreads / TPG;
  static constexpr int TRA = NT == 128 ? 16 : 32;                  // pass A rows per tile
  static constexpr int BUFA = TRA * NT * 20;                        // bytes: HA, Z (8 B), X (4 B)
  static constexpr int NJ = NT / 4, NI = kThreads / NJ, MR = 2, TRB = NI * MR;   // pass B
  static constexpr int LDT = NT + 2;                                // df32 row stride of T
  static constexpr int BUFB = TRB * NT * 24;                        // HA, Z, D (8 B each)
  static constexpr bool B_ASYNC = NT <= 64;                         // NT = 128: synchronous passB
  static constexpr int RED = RG > 1 ? RG * NT * NT * 8 : 0;        // cross-group reduction
  static constexpr int bytes_a = 2 * BUFA > RED ? 2 * BUFA : RED;
  static constexpr int bytes_b = NT * LDT * 8 + 2 * BUFB;
  static constexpr int bytes = B_ASYNC ? (bytes_a > bytes_b ? bytes_a : bytes_b) : bytes_a;
};

template <int NT>
__device__ void refreshA_async(const df32* __restrict__ HAdf, df32* Zdf, const float* __restrict__ X,
                               int64_t row0, int64_t row1, int N, unsigned char* tiles, double* __restrict__ out) {
  using TL = DFTile<NT>;
  constexpr int MA = TL::MA, NG = TL::NG, TPG = TL::TPG, RG = TL::RG, TR = TL::TRA;
  const int t = threadIdx.x, g = t / TPG, u = t % TPG, tj = u % NG, tk = u / NG;
  const int k0 = tk * MA, j0 = tj * MA;
  DFAcc acc[MA][MA];
  int since = 0;   // rows added since the last renormalisation
  auto issue = [&](int64_t i0, int b) {
    unsigned char* sb = tiles + b * TL::BUFA;
    df32* sH = reinterpret_cast<df32*>(sb);
    df32* sZ = sH + TR * NT;
    float* sX = reinterpret_cast<float*>(sZ + TR * NT);
    // HA and Z rows: 2 df32 per 16 bytes; X rows: 4 floats per 16 bytes
    for (int c = t; c < TR * (NT / 2); c += kThreads) {
      const int ii = c / (NT / 2), c0 = (c % (NT / 2)) * 2;
      const int64_t i = i0 + ii;
      const bool ok = i < row1 && c0 < N;
      const int64_t off = ok ? i * N + c0 : row0 * N;
      cp_async16(sH + ii * NT + c0, HAdf + off, ok);
      cp_async16(sZ + ii * NT + c0, Zdf + off, ok);
    }
    for (int c = t; c < TR * (NT / 4); c += kThreads) {
      const int ii = c / (NT / 4), c0 = (c % (NT / 4)) * 4;
      const int64_t i = i0 + ii;
      const bool ok = i < row1 && c0 < N;
      cp_async16(sX + ii * NT + c0, X + (ok ? i * N + c0 : row0 * N), ok);
    }
    cp_async_commit();
  };
  int b = 0;
  if (row0 < row1) issue(row0, 0);
  for (int64_t i0 = row0; i0 < row1; i0 += TR, b ^= 1) {
    if (i0 + TR < row1) {
      issue(i0 + TR, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    unsigned char* sb = tiles + b * TL::BUFA;
    const df32* sH = reinterpret_cast<const df32*>(sb);
    df32* sZ = reinterpret_cast<df32*>(sb) + TR * NT;
    const float* sX = reinterpret_cast<const float*>(sZ + TR * NT);
    // Z += X in the tile (and back to global)
    const int nrows = (int)imin64(TR, row1 - i0);
    for (int e = t; e < nrows * (N / 2); e += kThreads) {
      const int ii = e / (N / 2), c0 = (e % (N / 2)) * 2;
      const df32 z0 = sZ[ii * NT + c0] + df32(sX[ii * NT + c0], 0.f);
      const df32 z1 = sZ[ii * NT + c0 + 1] + df32(sX[ii * NT + c0 + 1], 0.f);
      sZ[ii * NT + c0] = z0;
      sZ[ii * NT + c0 + 1] = z1;
      *reinterpret_cast<float4*>(Zdf + (i0 + ii) * N + c0) = make_float4(z0.hi, z0.lo, z1.hi, z1.lo);
    }
    __syncthreads();
    for (int ii = g; ii < nrows; ii += RG) {
      df32 a[MA], v[MA];
      load_vec<df32>(a, sH + ii * NT + k0, MA);
      load_vec<df32>(v, sZ + ii * NT + j0, MA);
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) acc[x][y].add(a[x], v[y]);
      if (++since == 4) {
        since = 0;
#pragma unroll
        for (int x = 0; x < MA; ++x)
#pragma unroll
          for (int y = 0; y < MA; ++y) acc[x][y].renorm();
      }
    }
    __syncthreads();   // the buffer is refilled by the copy issued in the next iteration
  }
  double* red = reinterpret_cast<double*>(tiles);
  if (RG > 1) {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) red[(g * NT + k0 + x) * NT + j0 + y] = (double)acc[x][y].value();
    __syncthreads();
    if (g == 0) {
#pragma unroll
      for (int x = 0; x < MA; ++x)
#pragma unroll
        for (int y = 0; y < MA; ++y) {
          const int k = k0 + x, j = j0 + y;
          double s = 0.0;
          for (int gg = 0; gg < RG; ++gg) s += red[(gg * NT + k) * NT + j];
          if (k < N && j < N) out[k * N + j] = s;
        }
    }
  } else {
#pragma unroll
    for (int x = 0; x < MA; ++x)
#pragma unroll
      for (int y = 0; y < MA; ++y) {
        const int k = k0 + x, j = j0 + y;
        if (k < N && j < N) out[k * N + j] = (double)acc[x][y].value();
      }
  }
  if (t < N) {
    out[N * N + t] = 0.0;
    out[N * N + N + t] = 0.0;
  }
  __syncthreads();
}

// Pass B: B = hi(D - (r Z + HA T')) with T' = T/(N-1) staged in double-float (sT, stride
// LDT), rr_out[j] = block sum of the squared new residual (the float hi parts, as
// EpiRefreshDF). MR = 2 rows x 4 columns per thread.
template <int NT, typename VT>
__device__ void refreshB_async(const df32* __restrict__ HAdf, const df32* __restrict__ Zdf,
                               const df32* __restrict__ Ddf, const double* __restrict__ r, VT* B,
                               int64_t row0, int64_t row1, int N, const df32* sT, df32 inv,
                               unsigned char* tiles, double* rr_out) {
  using TL = DFTile<NT>;
  constexpr int NJ = TL::NJ, MR = TL::MR, TR = TL::TRB, LDT = TL::LDT;
  const int t = threadIdx.x, tj = t % NJ, ti = t / NJ, j0 = 4 * tj, r0 = ti * MR;
  float rr[4] = {0.f, 0.f, 0.f, 0.f};
  auto issue = [&](int64_t i0, int b) {
    unsigned char* sb = tiles + b * TL::BUFB;
    df32* sH = reinterpret_cast<df32*>(sb);
    df32* sZ = sH + TR * NT;
    df32* sD = sZ + TR * NT;
    for (int c = t; c < TR * (NT / 2); c += kThreads) {
      const int ii = c / (NT / 2), c0 = (c % (NT / 2)) * 2;
      const int64_t i = i0 + ii;
      const bool ok = i < row1 && c0 < N;
      const int64_t off = ok ? i * N + c0 : row0 * N;
      cp_async16(sH + ii * NT + c0, HAdf + off, ok);
      cp_async16(sZ + ii * NT + c0, Zdf + off, ok);
      cp_async16(sD + ii * NT + c0, Ddf + off, ok);
    }
    cp_async_commit();
  };
  int b = 0;
  if (row0 < row1) issue(row0, 0);
  for (int64_t i0 = row0; i0 < row1; i0 += TR, b ^= 1) {
    if (i0 + TR < row1) {
      issue(i0 + TR, b ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    unsigned char* sb = tiles + b * TL::BUFB;
    const df32* sH = reinterpret_cast<const df32*>(sb);
    const df32* sZ = sH + TR * NT;
    const df32* sD = sZ + TR * NT;
    DFAcc acc[MR][4];
    for (int k = 0; k < NT; k += 4) {   // NT % 4 == 0; renormalised after every 4 terms
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        df32 a[MR], bv[4];
#pragma unroll
        for (int x = 0; x < MR; ++x) a[x] = sH[(r0 + x) * NT + k + kk];
        load_vec<df32>(bv, sT + (k + kk) * LDT + j0, 4);
#pragma unroll
        for (int x = 0; x < MR; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y].add(a[x], bv[y]);
      }
#pragma unroll
      for (int x = 0; x < MR; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y].renorm();
    }
#pragma unroll
    for (int x = 0; x < MR; ++x) {
      const int64_t i = i0 + r0 + x;
      if (i < row1 && j0 < N) {
        const df32 ri(r[i]);
        df32 z[4], d[4];
        load_vec<df32>(z, sZ + (r0 + x) * NT + j0, 4);
        load_vec<df32>(d, sD + (r0 + x) * NT + j0, 4);
        VT o[4];
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const df32 q = fma(ri, z[y], acc[x][y].value() * inv);
          const df32 rt = d[y] - q;
          rr[y] = __fmaf_rn(rt.hi, rt.hi, rr[y]);
          o[y] = (VT)rt.hi;
        }
        st4<VT>(B + i * N, j0, N, true, o);
      }
    }
    __syncthreads();
  }
  double* red = reinterpret_cast<double*>(tiles);
#pragma unroll
  for (int y = 0; y < 4; ++y) red[ti * NT + j0 + y] = (double)rr[y];
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < TL::NI; ++q) s += red[q * NT + t];
    rr_out[t] = s;
  }
  __syncthreads();
}

// Compensated sum of squares of FP32 values (exact products by FMA, two-sum accumulation):
// the FP64 column norms of the FP32 T without FP64 arithmetic per term.
struct SqAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float ph = __fmul_rn(v, v);
    const float pl = __fmaf_rn(v, v, -ph);
    float t, e;
    df_two_sum(s, ph, t, e);
    s = t;
    c = __fadd_rn(c, __fadd_rn(e, pl));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Stage the reduced N x N matrix T (first N*N entries of Tred: FP64, or FP32 when CT is float,
// see reduce_slice) into shared memory as CT with stride NT + 16/sizeof(CT), zero-padded, and
// return the column norms ||T_:j||^2 of the staged T in tn2[j] (FP64 products for FP64, an
// exact-product compensated sum for FP32; thread j owns column j's sum over its rows; fixed
// order).
template <typename CT, int NT>
__device__ __forceinline__ void stage_T_norms(const double* __restrict__ Tred, int N, CT* sT,
                                              double* tn2, double* scratch) {
  constexpr int LD = NT + 16 / (int)sizeof(CT), L = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, k0 = t / NT;
  double nrm = 0.0;
  if constexpr (sizeof(CT) == 4) {
    const float* T32 = reinterpret_cast<const float*>(Tred);
    SqAcc acc;
    for (int k = k0; k < NT; k += L) {
      const float v = (k < N && j < N) ? __ldcg(T32 + k * N + j) : 0.f;
      sT[k * LD + j] = v;
      acc.add(v);
    }
    nrm = acc.value();
  } else {
    for (int k = k0; k < NT; k += L) {
      const double v = (k < N && j < N) ? __ldcg(Tred + k * N + j) : 0.0;
      sT[k * LD + j] = (CT)v;
      nrm = fma(v, v, nrm);
    }
  }
  for (int k = t; k < NT * (LD - NT); k += kThreads) sT[(k / (LD - NT)) * LD + NT + k % (LD - NT)] = CT(0);
  scratch[t] = nrm;
  __syncthreads();
  if (t < NT) {
    double s = 0.0;
    for (int q = 0; q < L; ++q) s += scratch[q * NT + t];
    tn2[t] = s;
  }
  __syncthreads();
}

// Stage T_{k+1} = Tz + beta_j T_k into shared memory in place (Tz: the reduced HA^T z_{k+1},
// FP32 at the start of Tred; sT holds T_k, stride NT + 4, zero-padded; with beta_j = 0, T_k is
// not read) and return the column norms ||T_{k+1,:j}||^2 (exact-product compensated FP32
// sums, fixed order). With `step` set, beta_j = gamma_{k+1}/gamma_k is formed here for the
// active columns from the reduced column sums [(r, z) | (r, r) | sum r_i z^2 | sum r_i z p]
// behind Tz, by every thread that stages a piece of column j (so the sums and Tz are read in
// one round), and the column's scalars are advanced: s_den = sum r_i p^2, s_sig = gamma,
// s_gam = (r, r), iteration count; beta (FP32) lands in beta[] for the next pass. Without
// `step`, beta[] is read as given.
template <int NT>
__device__ __forceinline__ void stage_T_rec(const double* __restrict__ Tred, int N, float* beta,
                                            float* sT, double* tn2, double* scratch, bool step = false,
                                            const int* s_active = nullptr, double* s_sig = nullptr,
                                            double* s_den = nullptr, double* s_gam = nullptr,
                                            int* s_iters = nullptr) {
  constexpr int LD = NT + 4, L = kThreads / NT;
  const int t = threadIdx.x, j = t % NT, k0 = t / NT;
  const float* T32 = reinterpret_cast<const float*>(Tred);
  float tz[NT / L];
#pragma unroll
  for (int q = 0; q < NT / L; ++q) {
    const int k = k0 + q * L;
    tz[q] = (k < N && j < N) ? __ldcg(T32 + k * N + j) : 0.f;
  }
  float bj = 0.f;
  double g1 = 0.0;
  const bool act = step && j < N && s_active[j];
  if (act) {
    g1 = __ldcg(Tred + N * N + j);
    bj = (float)(g1 / s_sig[j]);
  } else if (!step && j < N) {
    bj = beta[j];
  }
  SqAcc acc;
#pragma unroll
  for (int q = 0; q < NT / L; ++q) {
    const int k = k0 + q * L;
    // beta == 0 (a new inner solve, frozen columns) takes Tz without reading the old T: the
    // region may hold other passes' bytes, and 0 * NaN would not be 0
    const float v = (bj == 0.f) ? tz[q] : fmaf(bj, sT[k * LD + j], tz[q]);
    sT[k * LD + j] = v;
    acc.add(v);
  }
  for (int k = t; k < NT * (LD - NT); k += kThreads) sT[(k / (LD - NT)) * LD + NT + k % (LD - NT)] = 0.f;
  scratch[t] = acc.value();
  __syncthreads();   // every read of s_sig above precedes the updates below
  if (t < NT) {
    double sum = 0.0;
    for (int q = 0; q < L; ++q) sum += scratch[q * NT + t];
    tn2[t] = sum;
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
}

// Inner-solve set-up pass A: Res = B, X = 0, and V = B (preconditioned: V = B / r) for
// the first reduction.
template <typename VT, bool PC>
struct ProSetup {
  const VT* B;
  VT* X;
  VT* Res;
  const VT* rv;
  int N;
  __device__ __forceinline__ void operator()(int64_t i, int j0, VT (&v)[4], bool vec) {
    ld4<VT>(v, B + i * N, j0, N, vec);
    const VT z[4] = {VT(0), VT(0), VT(0), VT(0)};
    st4<VT>(X + i * N, j0, N, vec, z);
    st4<VT>(Res + i * N, j0, N, vec, v);
    if (PC) {
      const VT rinv = VT(1) / rv[i];
#pragma unroll
      for (int y = 0; y < 4; ++y) v[y] *= rinv;
    }
  }
};

// Refresh pass A (FP64): Z += X (refinement) and V = Z.
template <typename VT>
struct ProRefresh {
  double* Z;
  const VT* X;
  int N;
  bool accumulate;
  __device__ __forceinline__ void operator()(int64_t i, int j0, double (&v)[4], bool vec) {
    ld4<double>(v, Z + i * N, j0, N, vec);
    if (accumulate) {
      VT x[4];
      ld4<VT>(x, X + i * N, j0, N, vec);
#pragma unroll
      for (int y = 0; y < 4; ++y) v[y] += (double)x[y];
      st4<double>(Z + i * N, j0, N, vec, v);
    }
  }
};

// Refresh pass B (FP64): true residual D - (HA T/(N-1) + r Z); optionally the next
// right-hand side B = (VT) residual.
template <typename VT>
struct EpiRefresh {
  const double* Z;
  const double* D;
  const double* r;
  VT* B;
  double inv;
  int N;
  static constexpr bool kPrefetch = false;
  struct Frag { double z[4], d[4]; double ri; };
  __device__ __forceinline__ void prefetch(int64_t i, int j0, Frag& f, bool vec) {
    ld4<double>(f.z, Z + i * N, j0, N, vec);
    ld4<double>(f.d, D + i * N, j0, N, vec);
    f.ri = r[i];
  }
  __device__ __forceinline__ void apply(int64_t i, int j0, const double (&acc)[4], Frag& f,
                                        double (&rr)[4], bool vec) {
    double rt[4];
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const double q = fma(acc[y], inv, f.ri * f.z[y]);
      rt[y] = f.d[y] - q;
      rr[y] = fma(rt[y], rt[y], rr[y]);
    }
    if (B) {
      VT b[4];
#pragma unroll
      for (int y = 0; y < 4; ++y) b[y] = (VT)rt[y];
      st4<VT>(B + i * N, j0, N, vec, b);
    }
  }
};


// Double-float refresh, pass A: Z += X (X is the inner solve's correction, Z the solution in
// double-float) and V = Z, for T = HA^T Z.
template <typename VT>
struct ProRefreshDF {
  df32* Z;
  const VT* X;
  int N;
  bool accumulate;
  __device__ __forceinline__ void operator()(int64_t i, int j0, df32 (&v)[4], bool vec) {
    ld4<df32>(v, Z + i * N, j0, N, vec);
    if (accumulate) {
      VT x[4];
      ld4<VT>(x, X + i * N, j0, N, vec);
#pragma unroll
      for (int y = 0; y < 4; ++y) v[y] = v[y] + df32((float)x[y], 0.f);
      st4<df32>(Z + i * N, j0, N, vec, v);
    }
  }
};

// Double-float refresh, pass B: the true residual D - (HA T' + r Z) with T' = T/(N-1) staged
// in double-float; writes the next right-hand side B (float) and accumulates ||residual||^2.
template <typename VT>
struct EpiRefreshDF {
  const df32* Z;
  const df32* D;
  const double* r;
  VT* B;
  int N;
  df32 inv;   // 1/(N-1)
  static constexpr bool kPrefetch = false;
  struct Frag { df32 z[4], d[4]; df32 ri; };
  __device__ __forceinline__ void prefetch(int64_t i, int j0, Frag& f, bool vec) {
    ld4<df32>(f.z, Z + i * N, j0, N, vec);
    ld4<df32>(f.d, D + i * N, j0, N, vec);
    f.ri = df32(r[i]);
  }
  __device__ __forceinline__ void apply(int64_t i, int j0, const df32 (&acc)[4], Frag& f,
                                        df32 (&rr)[4], bool vec) {
    VT b[4];
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const df32 q = fma(f.ri, f.z[y], acc[y] * inv);
      const df32 rt = f.d[y] - q;
      rr[y].hi = __fmaf_rn(rt.hi, rt.hi, rr[y].hi);   // the norm only needs float accuracy
      b[y] = (VT)rt.hi;
    }
    if (B) st4<VT>(B + i * N, j0, N, vec, b);
  }
};

}  // namespace enkf
