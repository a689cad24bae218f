// Host side of the mixed-precision (BF16 / FP16 tensor-core) persistent solve: planning and
// launch. The kernels are in tc_mixed.cuh, instantiated by kernels_tc_bf16.cu and
// kernels_tc_fp16.cu.
#include <algorithm>

#include "tc_mixed.cuh"

namespace enkf {

void* mixed_kernel_bf16(bool pc, bool split, int NT);   // kernels_tc_bf16.cu
void* mixed_kernel_fp16(bool pc, bool split, int NT);   // kernels_tc_fp16.cu
static bool mixed_split(const enkf_config& c) { return c.lowprec_terms != 1; }
static void* mixed_select(const enkf_config& c, int NT) {
  const bool pc = c.precondition != 0;
  if (c.precision == ENKF_BF16_REFINE) return mixed_kernel_bf16(pc, mixed_split(c), NT);
  return mixed_kernel_fp16(pc, mixed_split(c), NT);
}
static size_t mixed_smem(int NT, bool split) {
  if (split) return NT == 32 ? mixed_smem_bytes<32, 3>() : (NT == 64 ? mixed_smem_bytes<64, 3>() : mixed_smem_bytes<128, 3>());
  return NT == 32 ? mixed_smem_bytes<32, 1>() : (NT == 64 ? mixed_smem_bytes<64, 1>() : mixed_smem_bytes<128, 1>());
}

cudaError_t plan_solve_mixed(enkf_handle_s* h) {
  const int N = h->cfg.N;
  const int NT = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
  void* fn = mixed_select(h->cfg, NT);
  const size_t smem = mixed_smem(NT, mixed_split(h->cfg));
  cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int occ = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem);
  if (err != cudaSuccess) return err;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // tensor memory: at most 512 columns per SM
  const int tmem_cap = 512 / (NT == 32 ? tc_tmem_cols<32>() : (NT == 64 ? tc_tmem_cols<64>() : tc_tmem_cols<128>()));
  occ = std::min(occ, tmem_cap);
  const int max_coresident = occ * h->sms;
  int G = (int)std::min<int64_t>(max_coresident, std::max<int64_t>(1, (h->cfg.m + kTR - 1) / kTR));
  if (h->cfg.grid_blocks > 0) G = std::min(h->cfg.grid_blocks, max_coresident);
  h->launch.G = G;
  h->launch.NT = NT;
  h->launch.smem = smem;
  return cudaSuccess;
}

// Tile images of HA for the tensor-core pass: tiles of 128 rows within each CTA's row block.
static int64_t mixed_rows_per(const enkf_handle_s* h) { return (h->cfg.m + h->launch.G - 1) / h->launch.G; }
static int mixed_qmax(const enkf_handle_s* h) { return (int)((mixed_rows_per(h) + kTR - 1) / kTR); }

size_t mixed_image_bytes(const enkf_handle_s* h) {
  const int TM = mixed_split(h->cfg) ? 2 : 1;
  return (size_t)h->launch.G * mixed_qmax(h) * TM * kTR * h->launch.NT * 2;
}

static cudaError_t launch_tc_images(enkf_handle_s* h) {
  const auto& c = h->cfg;
  const int blocks = (int)std::min<int64_t>((c.m * c.N + 255) / 256, (int64_t)h->sms * 32);
  const df32* HAdf = static_cast<const df32*>(h->ws.HAdf);
  const int64_t rp = mixed_rows_per(h);
  const int qm = mixed_qmax(h), NT = h->launch.NT;
  const bool split = mixed_split(c);
  if (c.precision == ENKF_BF16_REFINE) {
    auto* img = static_cast<__nv_bfloat16*>(h->ws.HA16);
    if (split) tc_images_kernel<__nv_bfloat16, 3><<<blocks, 256, 0, h->stream>>>(HAdf, c.m, c.N, NT, rp, qm, img, h->ws.hamax);
    else tc_images_kernel<__nv_bfloat16, 1><<<blocks, 256, 0, h->stream>>>(HAdf, c.m, c.N, NT, rp, qm, img, h->ws.hamax);
  } else {
    auto* img = static_cast<__half*>(h->ws.HA16);
    if (split) tc_images_kernel<__half, 3><<<blocks, 256, 0, h->stream>>>(HAdf, c.m, c.N, NT, rp, qm, img, h->ws.hamax);
    else tc_images_kernel<__half, 1><<<blocks, 256, 0, h->stream>>>(HAdf, c.m, c.N, NT, rp, qm, img, h->ws.hamax);
  }
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(enkf_handle_s* h) {
  const auto& c = h->cfg;
  auto& ws = h->ws;
  cudaError_t ierr = launch_tc_images(h);
  if (ierr != cudaSuccess) return ierr;
  MixedParams p{};
  p.m = c.m;
  p.N = c.N;
  p.HA16 = ws.HA16;
  p.qmax = mixed_qmax(h);
  p.HA32 = ws.HA32;
  p.HAdf = static_cast<const df32*>(ws.HAdf);
  p.Ddf = static_cast<const df32*>(ws.Ddf);
  p.Zdf = static_cast<df32*>(ws.Zdf);
  p.D = ws.D;
  p.B = static_cast<float*>(ws.B);
  p.r = ws.r;
  p.r32 = ws.r32;
  p.X = static_cast<float*>(ws.X);
  p.Res = static_cast<float*>(ws.Res);
  p.P = static_cast<float*>(ws.P);
  p.Sv = static_cast<float*>(ws.Sv);
  p.Tpart = ws.Tpart;
  p.Tred = ws.Tred;
  p.rrpart = ws.rrpart;
  p.W = ws.W;
  p.Tk = ws.Tk;
  p.Tacc = ws.Tacc;
  p.hamax = ws.hamax;
  p.zr = h->r_pow2;
  p.atomic_reduce = (c.reduce_order == 1 && h->launch.NT <= 64) ? 1 : 0;
  p.tol = c.tol;
  p.inner_tol = c.inner_tol;
  // accuracy an inner solve on the BF16 / FP16 operator can be asked for: the split FP16
  // operator with N <= 64 (each tile's Gram summed in FP32 outside the tensor cores) gains
  // about as much per inner solve as FP32 (512^2 / N = 64: 39 steps + 2 refreshes at 3e-5
  // against 47 + 3 at 1e-3); BF16 pairs carry 16 bits and N = 128 keeps the Gram in one TMEM
  // accumulator over all of a CTA's tiles, so those stay at 1e-3 (3 refreshes)
  const int nt_launch = h->launch.NT;
  p.itol_floor = mixed_split(c) ? ((c.precision == ENKF_FP16_REFINE && nt_launch <= 64) ? 3e-5 : 1e-3)
                                : (c.precision == ENKF_BF16_REFINE ? 2e-2 : 4e-3);
  p.max_iter = c.max_iter;
  p.refresh_every = c.refresh_every;
  p.col_iters = ws.col_iters;
  p.col_relres = ws.col_relres;
  p.col_true = ws.col_true;
  p.status = ws.status;
  p.bar = ws.bar;
  p.prof = h->prof_enabled ? ws.prof : nullptr;
  cudaError_t err = cudaMemsetAsync(ws.bar, 0, 4 * sizeof(unsigned), h->stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(ws.status, 0, 4 * sizeof(int32_t), h->stream);
  if (err != cudaSuccess) return err;
  void* fn = mixed_select(c, h->launch.NT);
  void* args[] = {&p};
  return cudaLaunchCooperativeKernel(fn, dim3(h->launch.G), dim3(kThreads), args, h->launch.smem, h->stream);
}

}  // namespace enkf
