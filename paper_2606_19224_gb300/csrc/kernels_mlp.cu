// Learned CG warm start: the MLP's forward, backward and Adam kernels, and the three
// warm-start maps of an analysis (features, prediction, decoder).
//
// The paper's CG starts from zero (Sec. 3.3). Every solution column of S Z = D satisfies
// R z_j = d_j - HA c_j with c_j = W e_j, W = HA^T Z/(N-1) (rearranging S Z = D with
// Eq. matvec_decomp), so the model predicts the N-vector c_j and the decoder forms
// z0_j = R^{-1}(d_j - HA c_j), whose residual lies in span(HA).
//
// Model (per column j): features f_j = [d_j(sketch)/s_j, g_j/s_j] with a sketch of K rows
// i_k = floor(k m / K), s_j the RMS of d_j over the sketch (1 if 0), g_j = HA^T R^-1 d_j/(N-1);
// standardised per feature; L hidden layers of width H with GELU (x Phi(x), Hendrycks &
// Gimpel 2016); linear output = standardised c_j/s_j. Loss: mean squared error in
// standardised units; optimiser: Adam (Kingma & Ba 2015, Algorithm 1).
//
// Parameter layout (FP32): per layer W [out][in] then b [out]; then mu_in [in], sd_in [in],
// mu_out [out], sd_out [out].
//
// The dense layers are FP32 SIMT tiles (64 x 64 outputs per 256-thread CTA, K-steps of 16
// staged in shared memory): the network is small (about 1.2 M weights) and its cost is a few
// microseconds per analysis, far below the solve; the forward kernel also serves training
// with a row gather and the input standardisation fused into its operand load.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "solve_body.cuh"

namespace enkf {

struct MlpLayout {
  int in, hidden, layers, out;
  int64_t w_off[8], b_off[8];   // per layer (layers + 1 <= 8)
  int64_t mu_in, sd_in, mu_out, sd_out, total, trained;
};

static bool mlp_layout(const enkf_mlp_shape* s, MlpLayout& L) {
  if (!s || s->in_dim < 1 || s->hidden < 1 || s->layers < 1 || s->layers > 7 || s->out_dim < 1) return false;
  L.in = s->in_dim;
  L.hidden = s->hidden;
  L.layers = s->layers;
  L.out = s->out_dim;
  int64_t off = 0;
  for (int l = 0; l <= L.layers; ++l) {
    const int64_t fi = l == 0 ? L.in : L.hidden, fo = l == L.layers ? L.out : L.hidden;
    L.w_off[l] = off;
    off += fi * fo;
    L.b_off[l] = off;
    off += fo;
  }
  L.trained = off;
  L.mu_in = off;
  off += L.in;
  L.sd_in = off;
  off += L.in;
  L.mu_out = off;
  off += L.out;
  L.sd_out = off;
  off += L.out;
  L.total = off;
  return true;
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// ------------------------------------------------------------------ tiled FP32 GEMM
// C[M][N] = sum_k A(m, k) B(k, n) with A(m, k) = A[m * sam + k * sak] and
// B(k, n) = B[k * sbk + n * sbn], and a fused epilogue.
constexpr int GBM = 64, GBN = 64, GBK = 32;

enum : int { EPI_HIDDEN = 0, EPI_OUT = 1, EPI_BWD = 2, EPI_STORE = 3 };

struct GemmArgs {
  const float* A;
  int64_t sam, sak;
  const float* B;
  int64_t sbk, sbn;
  int M, N, K;
  const float* bias;     // EPI_HIDDEN / EPI_OUT
  const float* zprev;    // EPI_BWD: pre-activations whose GELU' scales the product
  float* C;              // main output [M][N]
  float* C2;             // EPI_HIDDEN: GELU(C); EPI_OUT: raw output mu_out + sd_out * C
  const float* mu_out;
  const float* sd_out;
};

// TM x TM outputs per thread, (16 TM) x (16 TM) per CTA: TM = 4 for large products, TM = 2
// when the 64 x 64 grid would leave most SMs idle (the per-analysis inference, batch N).
template <int EPI, int TM>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(const GemmArgs g) {
  constexpr int BM = 16 * TM, BN = 16 * TM;
  __shared__ float As[GBK][BM + 4];
  __shared__ float Bs[GBK][BN + 4];
  const int t = threadIdx.x, tx = t % 16, ty = t / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  float acc[TM][TM] = {};
  // the next k-step's operands are loaded into registers while the current one is computed
  constexpr int LA = BM * GBK / 256, LB = GBK * BN / 256;
  float ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = t + q * 256, mm = e / GBK, kk = e % GBK;
      const int m = m0 + mm, k = k0 + kk;
      ra[q] = (m < g.M && k < g.K) ? g.A[(int64_t)m * g.sam + (int64_t)k * g.sak] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = t + q * 256, kk = e / BN, nn = e % BN;
      const int k = k0 + kk, n = n0 + nn;
      rb[q] = (k < g.K && n < g.N) ? g.B[(int64_t)k * g.sbk + (int64_t)n * g.sbn] : 0.f;
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int e = t + q * 256;
      As[e % GBK][e / GBK] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int e = t + q * 256;
      Bs[e / BN][e % BN] = rb[q];
    }
    __syncthreads();
    if (k0 + GBK < g.K) fetch(k0 + GBK);
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      float a[TM], b[TM];
#pragma unroll
      for (int x = 0; x < TM; ++x) a[x] = As[kk][ty * TM + x];
#pragma unroll
      for (int y = 0; y < TM; ++y) b[y] = Bs[kk][tx * TM + y];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TM; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int x = 0; x < TM; ++x) {
    const int m = m0 + ty * TM + x;
    if (m >= g.M) continue;
#pragma unroll
    for (int y = 0; y < TM; ++y) {
      const int n = n0 + tx * TM + y;
      if (n >= g.N) continue;
      const int64_t e = (int64_t)m * g.N + n;
      float v = acc[x][y];
      if (EPI == EPI_HIDDEN) {
        v += g.bias[n];
        g.C[e] = v;
        g.C2[e] = gelu_f(v);
      } else if (EPI == EPI_OUT) {
        v += g.bias[n];
        g.C[e] = v;
        if (g.C2) g.C2[e] = g.mu_out[n] + g.sd_out[n] * v;
      } else if (EPI == EPI_BWD) {
        g.C[e] = v * gelu_grad_f(g.zprev[e]);
      } else {
        g.C[e] = v;
      }
    }
  }
}

template <int EPI>
static cudaError_t gemm(const GemmArgs& a, cudaStream_t s) {
  const int64_t big = (int64_t)((a.N + GBN - 1) / GBN) * ((a.M + GBM - 1) / GBM);
  if (big >= 128) {
    dim3 grid((a.N + GBN - 1) / GBN, (a.M + GBM - 1) / GBM);
    mlp_gemm_kernel<EPI, 4><<<grid, 256, 0, s>>>(a);
  } else {
    dim3 grid((a.N + 31) / 32, (a.M + 31) / 32);
    mlp_gemm_kernel<EPI, 2><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Column sums of G [rows][cols] (the bias gradients), fixed order.
__global__ void colsum_kernel(const float* __restrict__ G, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += G[(int64_t)r * cols + c];
  out[c] = s;
}

// Loss and output gradient: diff = y_std - (t - mu_out)/sd_out over B x out entries (rows of
// T optionally gathered); G = 2 diff/(B out); loss = sum diff^2/(B out). One CTA, fixed order.
__global__ void __launch_bounds__(256) mse_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                                  const int32_t* __restrict__ rows, int B, int out,
                                                  const float* __restrict__ mu_out,
                                                  const float* __restrict__ sd_out, float* __restrict__ G,
                                                  float* __restrict__ loss) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  const double inv = 1.0 / ((double)B * out);
  double s = 0.0;
  for (int64_t e = t; e < (int64_t)B * out; e += 256) {
    const int b = (int)(e / out), o = (int)(e % out);
    const int64_t row = rows ? (int64_t)rows[b] : (int64_t)b;
    const float tt = (T[row * out + o] - mu_out[o]) / sd_out[o];
    const float d = Y[e] - tt;
    G[e] = (float)(2.0 * inv) * d;
    s += (double)d * d;
  }
  red[t] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  if (t == 0 && loss) *loss = (float)(red[0] * inv);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t count, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// Per-column mean and standard deviation over `rows` rows (population form; 1 where 0).
__global__ void colstats_kernel(const float* __restrict__ X, int64_t rows, int cols, float* __restrict__ mu,
                                float* __restrict__ sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int64_t r = 0; r < rows; ++r) s += X[r * cols + c];
  const double mean = s / (double)rows;
  double q = 0.0;
  for (int64_t r = 0; r < rows; ++r) {
    const double d = X[r * cols + c] - mean;
    q += d * d;
  }
  const double sdv = sqrt(q / (double)rows);
  mu[c] = (float)mean;
  sd[c] = sdv > 0.0 ? (float)sdv : 1.f;
}

// Gather rows of X [*][in] through `rows` (identity if NULL) and standardise per feature.
__global__ void standardize_rows_kernel(const float* __restrict__ X, const int32_t* __restrict__ rows, int B,
                                        int in, const float* __restrict__ mu, const float* __restrict__ sd,
                                        float* __restrict__ Xs) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * in;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / in), k = (int)(e % in);
    const int64_t row = rows ? (int64_t)rows[b] : (int64_t)b;
    Xs[e] = (X[row * in + k] - mu[k]) / sd[k];
  }
}

// ------------------------------------------------------------------ MLP, host side
struct MlpWork {
  float* Xs;     // standardised (gathered) input [B][in]
  float* Z[8];   // pre-activations per hidden layer [B][H]
  float* A[8];   // activations per hidden layer [B][H]
  float* Y;      // standardised output [B][out]
  float* G0;     // gradient buffers [B][max(H, out)]
  float* G1;
};

static size_t mlp_work_floats(const MlpLayout& L, int B) {
  const size_t w = (size_t)std::max(L.hidden, L.out);
  return (size_t)B * L.in + (size_t)2 * L.layers * B * L.hidden + (size_t)B * L.out + 2 * (size_t)B * w;
}

static MlpWork carve(const MlpLayout& L, int B, float* base) {
  MlpWork W{};
  float* q = base;
  W.Xs = q; q += (size_t)B * L.in;
  for (int l = 0; l < L.layers; ++l) {
    W.Z[l] = q; q += (size_t)B * L.hidden;
    W.A[l] = q; q += (size_t)B * L.hidden;
  }
  W.Y = q; q += (size_t)B * L.out;
  const size_t w = (size_t)std::max(L.hidden, L.out);
  W.G0 = q; q += (size_t)B * w;
  W.G1 = q;
  return W;
}

static int ew_grid(int64_t count) { return (int)std::min<int64_t>(4096, std::max<int64_t>(1, (count + 255) / 256)); }

static cudaError_t mlp_forward_impl(const MlpLayout& L, const float* P, const float* X, const int32_t* rows,
                                    int B, const MlpWork& W, float* Yraw, cudaStream_t s) {
  standardize_rows_kernel<<<ew_grid((int64_t)B * L.in), 256, 0, s>>>(X, rows, B, L.in, P + L.mu_in, P + L.sd_in, W.Xs);
  cudaError_t e = cudaGetLastError();
  for (int l = 0; l <= L.layers && e == cudaSuccess; ++l) {
    const int fi = l == 0 ? L.in : L.hidden, fo = l == L.layers ? L.out : L.hidden;
    GemmArgs a{};
    a.A = l == 0 ? W.Xs : W.A[l - 1];
    a.sam = fi;
    a.sak = 1;
    a.B = P + L.w_off[l];   // B(k, n) = W_l[n][k]
    a.sbk = 1;
    a.sbn = fi;
    a.M = B;
    a.N = fo;
    a.K = fi;
    a.bias = P + L.b_off[l];
    if (l < L.layers) {
      a.C = W.Z[l];
      a.C2 = W.A[l];
      e = gemm<EPI_HIDDEN>(a, s);
    } else {
      a.C = W.Y;
      a.C2 = Yraw;
      a.mu_out = P + L.mu_out;
      a.sd_out = P + L.sd_out;
      e = gemm<EPI_OUT>(a, s);
    }
  }
  return e;
}

static cudaError_t mlp_loss_grad_impl(const MlpLayout& L, const float* P, const float* X, const float* T,
                                      const int32_t* rows, int B, float* grad, float* loss, const MlpWork& W,
                                      cudaStream_t s) {
  cudaError_t e = mlp_forward_impl(L, P, X, rows, B, W, nullptr, s);
  if (e != cudaSuccess) return e;
  mse_kernel<<<1, 256, 0, s>>>(W.Y, T, rows, B, L.out, P + L.mu_out, P + L.sd_out, W.G0, loss);
  e = cudaGetLastError();
  float* g = W.G0;    // dL/dz of layer l, [B][fo]
  float* gn = W.G1;
  for (int l = L.layers; l >= 0 && e == cudaSuccess; --l) {
    const int fi = l == 0 ? L.in : L.hidden, fo = l == L.layers ? L.out : L.hidden;
    // dW_l[o][i] = sum_b g[b][o] a_{l-1}[b][i]
    GemmArgs a{};
    a.A = g;
    a.sam = 1;
    a.sak = fo;
    a.B = l == 0 ? W.Xs : W.A[l - 1];
    a.sbk = fi;
    a.sbn = 1;
    a.M = fo;
    a.N = fi;
    a.K = B;
    a.C = grad + L.w_off[l];
    e = gemm<EPI_STORE>(a, s);
    if (e != cudaSuccess) break;
    colsum_kernel<<<(fo + 255) / 256, 256, 0, s>>>(g, B, fo, grad + L.b_off[l]);
    e = cudaGetLastError();
    if (l > 0 && e == cudaSuccess) {
      // g_{l-1}[b][i] = (sum_o g[b][o] W_l[o][i]) GELU'(z_{l-1}[b][i])
      GemmArgs d{};
      d.A = g;
      d.sam = fo;
      d.sak = 1;
      d.B = P + L.w_off[l];
      d.sbk = fi;
      d.sbn = 1;
      d.M = B;
      d.N = fi;
      d.K = fo;
      d.zprev = W.Z[l - 1];
      d.C = gn;
      e = gemm<EPI_BWD>(d, s);
      std::swap(g, gn);
    }
  }
  return e;
}

// ------------------------------------------------------------------ warm-start maps
// Partial N x N products over row blocks: part[b][0][k][j] = sum_{i in block b} HA[i][k] D[i][j] / r_i
// and part[b][1][k][j] = sum_{i in block b} HA[i][k] HA[i][j] / r_i (FP32 products of the FP32
// copies, FP32 within a block); the reduce kernel sums the blocks in a fixed order in FP64.
// AM x AM outputs of each product per thread (AM = NT / 16).
constexpr int kWarmRows = 32;

template <int AM>
__global__ void __launch_bounds__(kThreads) warm_gram_kernel(const float* __restrict__ HA,
                                                             const double* __restrict__ D,
                                                             const float* __restrict__ r32, int64_t m, int N,
                                                             int64_t rows_per, double* __restrict__ part) {
  constexpr int NT = 16 * AM, LD = NT + 4, RW = AM == 8 ? kWarmRows / 2 : kWarmRows;   // static smem < 48 KB
  __shared__ __align__(16) float sH[RW][LD];
  __shared__ __align__(16) float sD[RW][LD];
  __shared__ __align__(16) float sHr[RW][LD];
  __shared__ float sRi[RW];
  const int t = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * rows_per, i1 = imin64(m, i0 + rows_per);
  // thread (tk, tj) owns the AM x AM block k in [AM tk, AM tk + AM), j in [AM tj, AM tj + AM)
  const int tk = t / 16, tj = t % 16, k0 = AM * tk, c0 = AM * tj;
  float acc[AM][AM] = {}, accG[AM][AM] = {};
  for (int64_t ib = i0; ib < i1; ib += RW) {
    __syncthreads();
    if (t < RW) {
      const int64_t i = ib + t;
      sRi[t] = i < i1 ? 1.f / r32[i] : 0.f;
    }
    __syncthreads();
    for (int e = t; e < RW * NT; e += kThreads) {
      const int ii = e / NT, k = e % NT;
      const int64_t i = ib + ii;
      const bool in = i < i1 && k < N;
      const float rinv = sRi[ii];
      const float h = in ? HA[i * N + k] : 0.f;
      sH[ii][k] = h;
      sHr[ii][k] = h * rinv;
      sD[ii][k] = in ? (float)D[i * N + k] * rinv : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < RW; ++ii) {
      float h[AM], d[AM], hr[AM];
#pragma unroll
      for (int a = 0; a < AM; a += 2) {
        const float2 v = *reinterpret_cast<const float2*>(&sH[ii][k0 + a]);
        h[a] = v.x;
        h[a + 1] = v.y;
        const float2 w = *reinterpret_cast<const float2*>(&sD[ii][c0 + a]);
        d[a] = w.x;
        d[a + 1] = w.y;
        const float2 q = *reinterpret_cast<const float2*>(&sHr[ii][c0 + a]);
        hr[a] = q.x;
        hr[a + 1] = q.y;
      }
#pragma unroll
      for (int a = 0; a < AM; ++a)
#pragma unroll
        for (int c = 0; c < AM; ++c) {
          acc[a][c] = fmaf(h[a], d[c], acc[a][c]);
          accG[a][c] = fmaf(h[a], hr[c], accG[a][c]);
        }
    }
  }
  double* out = part + (int64_t)blockIdx.x * 2 * N * N;
#pragma unroll
  for (int a = 0; a < AM; ++a)
#pragma unroll
    for (int c = 0; c < AM; ++c) {
      const int k = k0 + a, j = c0 + c;
      if (k < N && j < N) {
        out[k * N + j] = acc[a][c];
        out[N * N + k * N + j] = accG[a][c];
      }
    }
}

// g[k][j] = sum over the row-block partials in block order (one thread per entry).
__global__ void warm_reduce_kernel(const double* __restrict__ part, int nparts, int NN, double* __restrict__ g) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NN) return;
  double s = 0.0;
#pragma unroll 8
  for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * NN + e];
  g[e] = s;
}

// Features of column j (one CTA per column): sketch values, their RMS s_j, and g_j/s_j.
__global__ void __launch_bounds__(kThreads) warm_features_kernel(const double* __restrict__ D, int64_t m, int N,
                                                                 int K, const double* __restrict__ gsum,
                                                                 float* __restrict__ F,
                                                                 float* __restrict__ s_out) {
  __shared__ double red[kThreads];
  const int j = blockIdx.x, t = threadIdx.x;
  const double inv_nm1 = 1.0 / (double)(N - 1);
  double q = 0.0;
  for (int k = t; k < K; k += kThreads) {
    const int64_t i = ((int64_t)k * m) / K;
    const double v = D[i * N + j];
    q += v * v;
  }
  red[t] = q;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  const double rms = sqrt(red[0] / (double)K);
  const double sj = rms > 0.0 ? rms : 1.0;
  const int in = K + N;
  for (int k = t; k < K; k += kThreads) {
    const int64_t i = ((int64_t)k * m) / K;
    F[(int64_t)j * in + k] = (float)(D[i * N + j] / sj);
  }
  for (int k = t; k < N; k += kThreads) F[(int64_t)j * in + K + k] = (float)(gsum[k * N + j] * inv_nm1 / sj);
  if (t == 0) s_out[j] = (float)sj;
}

// Targets of the training pairs: T[j][k] = W[k][j] / s_j.
__global__ void warm_targets_kernel(const double* __restrict__ W, const float* __restrict__ s, int N,
                                    float* __restrict__ T) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int j = e / N, k = e % N;
  T[e] = (float)(W[k * N + j] / (double)s[j]);
}

// Coefficients of column j (one CTA per column): c_j = Y[j] s_j (the prediction in raw units)
// and e_j = c_j + (Gw c_j - g~_j)/(N-1) with Gw = HA^T R^-1 HA, g~_j = HA^T R^-1 d_j, so that the
// start z0_j = R^-1 (d_j - HA c_j) has residual d_j - S z0_j = HA e_j (from S = HA HA^T/(N-1) + R).
__global__ void __launch_bounds__(128) warm_coef_kernel(const float* __restrict__ Y, const float* __restrict__ s,
                                                        const double* __restrict__ gsum, int N,
                                                        float* __restrict__ C, float* __restrict__ Ecoef) {
  __shared__ double sc[128];
  const int j = blockIdx.x, t = threadIdx.x;
  const double sj = s[j];
  for (int k = t; k < N; k += 128) sc[k] = (double)Y[j * N + k] * sj;
  __syncthreads();
  const double* g = gsum;                 // [k][j] = HA^T R^-1 D
  const double* Gw = gsum + N * N;        // [k][l] = HA^T R^-1 HA
  const double inv = 1.0 / (double)(N - 1);
  for (int k = t; k < N; k += 128) {
    double acc = 0.0;
    for (int l = 0; l < N; ++l) acc = fma(Gw[k * N + l], sc[l], acc);
    C[k * N + j] = (float)sc[k];
    Ecoef[k * N + j] = (float)(sc[k] + (acc - g[k * N + j]) * inv);
  }
}

// Decoder: z0[i][j] = (d_ij - sum_k HA[i][k] C[k][j]) / r_i as the double-float starting solution
// of the FP32 solve, and its residual B[i][j] = sum_k HA[i][k] E[k][j] as the first inner
// right-hand side (FP32; the refreshes recompute the true residual in double-float).
template <int RB>
__global__ void __launch_bounds__(kThreads) warm_decode_kernel(const float* __restrict__ HA,
                                                               const double* __restrict__ D,
                                                               const float* __restrict__ r32, int64_t m, int N,
                                                               const float* __restrict__ C,
                                                               const float* __restrict__ Ecoef,
                                                               df32* __restrict__ Z0, float* __restrict__ B) {
  extern __shared__ float wsm[];   // C [N][N + 1], E [N][N + 1], a 16-row tile of HA [16][N + 1]
  const int LD = N + 1;
  float* sC = wsm;
  float* sE = wsm + N * LD;
  float* sHt = wsm + 2 * N * LD;
  const int t = threadIdx.x;
  for (int e = t; e < N * N; e += kThreads) {
    const int k = e / N, j = e % N;
    sC[k * LD + j] = C[e];
    sE[k * LD + j] = Ecoef[e];
  }
  // thread (column j, group g of RB consecutive rows of the 16-row block): the C and E entries
  // of column j are loaded once per k for RB rows (RB = 2, 4, 8 for N <= 32, 64, 128)
  for (int64_t ib = (int64_t)blockIdx.x * 16; ib < m; ib += (int64_t)gridDim.x * 16) {
    __syncthreads();
    for (int e = t; e < 16 * N; e += kThreads) {
      const int ii = e / N, k = e % N;
      const int64_t i = ib + ii;
      sHt[ii * LD + k] = i < m ? HA[i * N + k] : 0.f;
    }
    __syncthreads();
    constexpr int NGR = 16 / RB;   // row groups covering the 16 rows
    for (int e = t; e < N * NGR; e += kThreads) {
      const int j = e % N, g = e / N;
      float a1[RB], a2[RB];
#pragma unroll
      for (int x = 0; x < RB; ++x) { a1[x] = 0.f; a2[x] = 0.f; }
#pragma unroll 4
      for (int k = 0; k < N; ++k) {
        const float c = sC[k * LD + j], ev = sE[k * LD + j];
#pragma unroll
        for (int x = 0; x < RB; ++x) {
          const float h = sHt[(g * RB + x) * LD + k];
          a1[x] = fmaf(h, c, a1[x]);
          a2[x] = fmaf(h, ev, a2[x]);
        }
      }
#pragma unroll
      for (int x = 0; x < RB; ++x) {
        const int64_t i = ib + g * RB + x;
        if (i < m) {
          const float z = ((float)D[i * N + j] - a1[x]) / r32[i];
          Z0[i * N + j] = df32(z, 0.f);
          B[i * N + j] = a2[x];
        }
      }
    }
  }
}

}  // namespace enkf

// ------------------------------------------------------------------ host side
namespace enkf {

struct WarmState {
  MlpLayout L{};
  const float* params = nullptr;   // caller-owned model (enkf_set_warm_model)
  int K = 0;                       // sketch size of the model (in_dim - N)
  int nparts = 0;
  double* part = nullptr;          // [nparts][2][N][N]
  double* gsum = nullptr;          // [2][N][N]: HA^T R^-1 D, HA^T R^-1 HA
  float* C = nullptr;              // [N][N] predicted coefficients (column j = c_j)
  float* E = nullptr;              // [N][N] residual coefficients of the start
  float* F = nullptr;              // [N][K + N] features of the current analysis
  float* s = nullptr;              // [N] column scales
  float* Y = nullptr;              // [N][N] raw predictions
  float* work = nullptr;           // MLP activations for a batch of N rows
  int K_alloc = 0;
};

static cudaError_t warm_alloc(enkf_handle_s* h, int K) {
  if (!h->warm) h->warm = new WarmState();
  WarmState& w = *h->warm;
  const int N = h->cfg.N;
  cudaError_t e = cudaSuccess;
  if (!w.part) {
    w.nparts = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->sms, (h->cfg.m + 255) / 256));
    e = cudaMalloc((void**)&w.part, sizeof(double) * (size_t)w.nparts * 2 * N * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.gsum, sizeof(double) * 2 * N * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.C, sizeof(float) * N * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.E, sizeof(float) * N * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.s, sizeof(float) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w.Y, sizeof(float) * N * N);
  }
  if (e == cudaSuccess && K > w.K_alloc) {
    if (w.F) cudaFree(w.F);
    w.F = nullptr;
    e = cudaMalloc((void**)&w.F, sizeof(float) * (size_t)N * (K + N));
    if (e == cudaSuccess) w.K_alloc = K;
  }
  return e;
}

static cudaError_t warm_features_into(enkf_handle_s* h, int K, float* F) {
  WarmState& w = *h->warm;
  const auto& c = h->cfg;
  const int64_t rows_per = (c.m + w.nparts - 1) / w.nparts;
  if (c.N <= 32)
    warm_gram_kernel<2><<<w.nparts, kThreads, 0, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, rows_per, w.part);
  else if (c.N <= 64)
    warm_gram_kernel<4><<<w.nparts, kThreads, 0, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, rows_per, w.part);
  else
    warm_gram_kernel<8><<<w.nparts, kThreads, 0, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, rows_per, w.part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  warm_reduce_kernel<<<(2 * c.N * c.N + 255) / 256, 256, 0, h->stream>>>(w.part, w.nparts, 2 * c.N * c.N, w.gsum);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  warm_features_kernel<<<c.N, kThreads, 0, h->stream>>>(h->ws.D, c.m, c.N, K, w.gsum, F, w.s);
  return cudaGetLastError();
}

cudaError_t warm_features(enkf_handle_s* h, int K, float* F, float* T) {
  cudaError_t e = warm_alloc(h, 0);
  if (e == cudaSuccess) e = warm_features_into(h, K, F);
  if (e == cudaSuccess && T) {
    warm_targets_kernel<<<(h->cfg.N * h->cfg.N + 255) / 256, 256, 0, h->stream>>>(h->ws.W, h->warm->s, h->cfg.N, T);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t warm_set_model(enkf_handle_s* h, const enkf_mlp_shape* shape, const float* params, std::string& err) {
  MlpLayout L;
  if (!mlp_layout(shape, L)) { err = "bad MLP shape"; return cudaErrorInvalidValue; }
  const int N = h->cfg.N;
  if (L.out != N || L.in <= N) { err = "the model must map K + N features to N outputs (K >= 1)"; return cudaErrorInvalidValue; }
  cudaError_t e = warm_alloc(h, L.in - N);
  if (e != cudaSuccess) { err = "allocation"; return e; }
  WarmState& w = *h->warm;
  if (w.work) cudaFree(w.work);
  w.work = nullptr;
  e = cudaMalloc((void**)&w.work, sizeof(float) * mlp_work_floats(L, N));
  if (e != cudaSuccess) { err = "allocation"; return e; }
  const int smem = (int)(sizeof(float) * (size_t)(2 * N + 16) * (N + 1));   // up to 140 KB at N = 128
  e = cudaFuncSetAttribute(warm_decode_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(warm_decode_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(warm_decode_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) { err = "decoder shared memory"; return e; }
  w.L = L;
  w.params = params;
  w.K = L.in - N;
  return cudaSuccess;
}

bool warm_ready(const enkf_handle_s* h) { return h->warm && h->warm->params; }

// Learned start of one analysis: features -> MLP -> decoder into the solve's Zdf.
cudaError_t warm_prepare(enkf_handle_s* h) {
  WarmState& w = *h->warm;
  const auto& c = h->cfg;
  cudaError_t e = warm_features_into(h, w.K, w.F);
  if (e != cudaSuccess) return e;
  const MlpWork W = carve(w.L, c.N, w.work);
  e = mlp_forward_impl(w.L, w.params, w.F, nullptr, c.N, W, w.Y, h->stream);
  if (e != cudaSuccess) return e;
  warm_coef_kernel<<<c.N, 128, 0, h->stream>>>(w.Y, w.s, w.gsum, c.N, w.C, w.E);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = sizeof(float) * (size_t)(2 * c.N + 16) * (c.N + 1);
  const int grid = (int)std::min<int64_t>(2 * (int64_t)h->sms, (c.m + 15) / 16);
  df32* Z0 = static_cast<df32*>(h->ws.Zdf);
  float* B0 = static_cast<float*>(h->ws.B);
  if (c.N <= 32)
    warm_decode_kernel<2><<<grid, kThreads, smem, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, w.C, w.E, Z0, B0);
  else if (c.N <= 64)
    warm_decode_kernel<4><<<grid, kThreads, smem, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, w.C, w.E, Z0, B0);
  else
    warm_decode_kernel<8><<<grid, kThreads, smem, h->stream>>>(h->ws.HA32, h->ws.D, h->ws.r32, c.m, c.N, w.C, w.E, Z0, B0);
  return cudaGetLastError();
}

void warm_free(enkf_handle_s* h) {
  WarmState* w = h->warm;
  if (!w) return;
  void* ptrs[] = {w->part, w->gsum, w->C, w->E, w->F, w->s, w->Y, w->work};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete w;
  h->warm = nullptr;
}

int64_t mlp_param_count(const enkf_mlp_shape* s) {
  MlpLayout L;
  return mlp_layout(s, L) ? L.total : -1;
}

int64_t mlp_work_bytes(const enkf_mlp_shape* s, int B) {
  MlpLayout L;
  return (mlp_layout(s, L) && B > 0) ? (int64_t)(sizeof(float) * mlp_work_floats(L, B)) : -1;
}

cudaError_t mlp_forward(const enkf_mlp_shape* s, const float* P, const float* X, const int32_t* rows, int B,
                        float* Y, void* work, cudaStream_t st) {
  MlpLayout L;
  if (!mlp_layout(s, L) || B < 1) return cudaErrorInvalidValue;
  return mlp_forward_impl(L, P, X, rows, B, carve(L, B, static_cast<float*>(work)), Y, st);
}

cudaError_t mlp_loss_grad(const enkf_mlp_shape* s, const float* P, const float* X, const float* T,
                          const int32_t* rows, int B, float* grad, float* loss, void* work, cudaStream_t st) {
  MlpLayout L;
  if (!mlp_layout(s, L) || B < 1) return cudaErrorInvalidValue;
  return mlp_loss_grad_impl(L, P, X, T, rows, B, grad, loss, carve(L, B, static_cast<float*>(work)), st);
}

cudaError_t mlp_adam(int64_t count, float* P, const float* g, float* m, float* v, int step, float lr, float b1,
                     float b2, float eps, cudaStream_t st) {
  const float c1 = (float)(1.0 - std::pow((double)b1, step)), c2 = (float)(1.0 - std::pow((double)b2, step));
  adam_kernel<<<ew_grid(count), 256, 0, st>>>(P, g, m, v, count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_train_epoch(const enkf_mlp_shape* s, float* P, float* m, float* v, const float* X, const float* T,
                            const int32_t* perm, int64_t rows, int B, int step0, float lr, float* losses,
                            void* work, float* grad, cudaStream_t st) {
  MlpLayout L;
  if (!mlp_layout(s, L) || B < 1 || rows < B) return cudaErrorInvalidValue;
  const MlpWork W = carve(L, B, static_cast<float*>(work));
  cudaError_t e = cudaSuccess;
  const int64_t nb = rows / B;
  for (int64_t q = 0; q < nb && e == cudaSuccess; ++q) {
    e = mlp_loss_grad_impl(L, P, X, T, perm + q * B, B, grad, losses ? losses + q : nullptr, W, st);
    if (e == cudaSuccess) e = mlp_adam(L.trained, P, grad, m, v, step0 + (int)q + 1, lr, 0.9f, 0.999f, 1e-8f, st);
  }
  return e;
}

cudaError_t mlp_standardize(const enkf_mlp_shape* s, float* P, const float* X, const float* T, int64_t rows,
                            cudaStream_t st) {
  MlpLayout L;
  if (!mlp_layout(s, L) || rows < 1) return cudaErrorInvalidValue;
  colstats_kernel<<<(L.in + 127) / 128, 128, 0, st>>>(X, rows, L.in, P + L.mu_in, P + L.sd_in);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) colstats_kernel<<<(L.out + 127) / 128, 128, 0, st>>>(T, rows, L.out, P + L.mu_out, P + L.sd_out);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace enkf
