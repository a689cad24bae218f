// CUDA kernels of the CGD-EnKF analysis step on CUDA cores (FP64 and FP32 paths).
//
//   innov_kernel   Z_obs = H X_f (CSR gather), zbar, HA = Z_obs - zbar 1^T, E (Philox or given),
//                  D = y 1^T - Z_obs + E                         (Sec. 2.3, Eq. Zhat_def)
//   solve_kernel   persistent cooperative CG on S Z = D with S V = HA (HA^T V)/(N-1) + R V
//                  (Sec. 3.3, Eq. matvec_decomp); N independent recurrences share each
//                  matvec; FP64 scalars; FP32 mode = FP32 inner solves + double-float residual
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
#include "innov_device.cuh"
#include "solve_body.cuh"

#include <algorithm>

namespace enkf {

template <typename VT, int NT, bool PC>
__global__ void __launch_bounds__(kThreads, (NT == 128 || sizeof(VT) == 8 || async_passF<VT, NT>()) ? 1 : 2)
    solve_kernel(SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  GridBarrier bar{p.bar, reinterpret_cast<int*>(p.bar + 1), p.status, gridDim.x, 0u};
  solve_body<VT, NT, PC>(p, (int)gridDim.x, (int)blockIdx.x, bar, smem);
}

template <typename VT>
__global__ void __launch_bounds__(kThreads) innov_kernel(
    const VT* __restrict__ Xf, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const double* __restrict__ w, const double* __restrict__ y, const double* __restrict__ r,
    const double* __restrict__ E, int emode, uint64_t seed, uint64_t counter, int64_t m, int N,
    double* __restrict__ HA64, float* __restrict__ HA32, double* __restrict__ D,
    float* __restrict__ B32, __nv_bfloat16* __restrict__ HAb, __half* __restrict__ HAh,
    int split_lo, df32* __restrict__ HAdf, df32* __restrict__ Ddf, unsigned* hamax) {
  const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  innov_rows<VT>(Xf, rowptr, col, w, y, r, E, emode, seed, counter, m, N, HA64, HA32, D, B32, HAb,
                 HAh, split_lo, HAdf, Ddf, 0, m, warp, nwarps, hamax);
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

template <typename VT, int NT, int MODE = 0>
__global__ void __launch_bounds__(kThreads) update_kernel(const VT* Xf, VT* Xa,
                                                          const double* __restrict__ W,
                                                          int64_t n, int N) {
  extern __shared__ __align__(16) unsigned char smem[];
  update_rows<VT, NT, MODE>(Xf, Xa, W, n, N, blockIdx.x, gridDim.x, smem);
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
  // the tensor-core modes scale the HA image by a power of two from the largest |HA|
  if (ws.hamax) {
    cudaError_t e = cudaMemsetAsync(ws.hamax, 0, sizeof(unsigned), h->stream);
    if (e != cudaSuccess) return e;
  }
  if (fp64)
    innov_kernel<double><<<blocks, kThreads, 0, h->stream>>>(
        static_cast<const double*>(Xf), ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter,
        c.m, c.N, ws.HA64, nullptr, ws.D, nullptr, nullptr, nullptr, 0, nullptr, nullptr, nullptr);
  else
    innov_kernel<float><<<blocks, kThreads, 0, h->stream>>>(
        static_cast<const float*>(Xf), ws.rowptr, ws.col, ws.w, y, ws.r, E, emode, seed, counter,
        c.m, c.N, ws.HA64, ws.HA32, ws.D, static_cast<float*>(ws.B),
        nullptr, nullptr, 0, static_cast<df32*>(ws.HAdf), static_cast<df32*>(ws.Ddf), ws.hamax);
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
  p.warm = (h->cfg.warm_start && h->cfg.precision == ENKF_FP32) ? 1 : 0;
  p.warm_accept = h->cfg.warm_accept;
  p.col_warm = ws.col_warm;
  p.Tacc = ws.Tacc;
  // atomic step sums pay for N <= 64; at N = 128 the 16,384 atomic adds per CTA and step cost
  // more than the reduction they replace (1024^2 / N = 128: 37.5 -> 41.3 ms)
  p.atomic_reduce = (c.reduce_order == 1 && !fp64 && h->launch.NT <= 64) ? 1 : 0;
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
  // FP32 ensembles: the A W product on the tensor cores (kernels_update_tc.cu); FP64 on CUDA cores
  if (h->cfg.precision != ENKF_FP64) return launch_update_tc(h, Xf, Xa);
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
