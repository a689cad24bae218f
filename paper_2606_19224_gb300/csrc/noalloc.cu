// enkf_analyze_noalloc: one analysis step that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need an analysis: code that runs
// while a CUDA stream is being captured into a graph (an allocation there breaks or
// invalidates the capture), applications that hand all device memory to their own pool
// allocator up front and forbid later allocations, and real-time assimilation loops that
// must not touch the allocator after start-up. For them this entry point keeps all of its
// working memory in one file-scope device array of fixed size (kScratchBytes, below),
// which every GPU that loads the library holds until the process exits.
//
// The analysis is the same as enkf_create + enkf_analyze + enkf_get_stats (same kernels,
// same launch plan), with the observation operator and R passed as device pointers.
#include <cstring>
#include <mutex>

#include "common.cuh"

namespace {

// Fixed working memory of the no-allocation entry point: 16 MiB per device.
constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

enkf_status noalloc_fail(enkf_status s, const char* msg) {
  (void)msg;  // argument errors are reported by status code alone, as elsewhere in the ABI
  return s;
}

// Device address of g_scratch on the current device, looked up once per device (the
// symbol's host-side name is only a stand-in and must never be passed to a kernel).
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

enkf_status enkf_analyze_noalloc(const enkf_config* cfg, const int32_t* d_rowptr,
                                 const int32_t* d_col, const double* d_w, const double* d_r,
                                 const void* d_Xf, const double* d_y, uint64_t seed,
                                 uint64_t counter, void* d_Xa, void* cuda_stream,
                                 enkf_stats* out_stats) {
  if (!cfg || !d_rowptr || !d_r || !d_Xf || !d_y || !d_Xa)
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: NULL argument");
  const enkf_config c = *cfg;
  if (c.n < 1 || c.m < 1 || c.N < 2)
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: need n >= 1, m >= 1, N >= 2");
  if (c.m >= (int64_t(1) << 32) || c.n >= (int64_t(1) << 31))
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: m must be < 2^32 and n < 2^31");
  if (c.N > 128) return noalloc_fail(ENKF_ERR_UNSUPPORTED, "enkf_analyze_noalloc: N > 128");
  if (c.precision != ENKF_FP64 && c.precision != ENKF_FP32)
    return noalloc_fail(ENKF_ERR_UNSUPPORTED, "enkf_analyze_noalloc: precision must be FP64 or FP32");
  if (c.variant != ENKF_CGD)
    return noalloc_fail(ENKF_ERR_UNSUPPORTED, "enkf_analyze_noalloc: variant must be ENKF_CGD");
  if (c.warm_start != 0)
    return noalloc_fail(ENKF_ERR_UNSUPPORTED, "enkf_analyze_noalloc: no learned warm start (it needs a handle)");
  if (c.fixed_iters < 0 || c.max_iter < 1 || c.max_refine < 0 || c.grid_blocks < 0)
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: bad iteration limits");
  if (c.fixed_iters == 0 && !(c.tol > 0.0))
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: tol must be positive");
  if (c.precision == ENKF_FP32 && !(c.inner_tol > 0.0 && c.inner_tol < 1.0))
    return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: inner_tol must be in (0, 1)");
  {
    // X_a may be X_f itself (in-place) but must not partially overlap it: the update kernel
    // reads X_f rows while it writes X_a rows
    const size_t xb = (c.precision == ENKF_FP64 ? 8 : 4) * size_t(c.n) * size_t(c.N);
    const char* a = static_cast<const char*>(d_Xf);
    const char* b = static_cast<const char*>(d_Xa);
    if (a != b && a < b + xb && b < a + xb)
      return noalloc_fail(ENKF_ERR_INVALID_ARG, "enkf_analyze_noalloc: X_a partially overlaps X_f");
  }

  enkf_handle_s h;
  h.cfg = c;
  h.stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h.device);
  if (e == cudaSuccess && (h.device < 0 || h.device >= kMaxDevices)) e = cudaErrorInvalidDevice;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h.sms, cudaDevAttrMultiProcessorCount, h.device);
  if (e == cudaSuccess) e = enkf::plan_solve(&h);
  if (e != cudaSuccess) return noalloc_fail(ENKF_ERR_CUDA, "enkf_analyze_noalloc: planning");

  // carve the workspace out of the fixed array
  const size_t mN = size_t(c.m) * c.N;
  const size_t NE = size_t(c.N) * c.N + 4 * size_t(c.N);
  const bool fp64 = c.precision == ENKF_FP64;
  const size_t vs = fp64 ? 8 : 4;
  struct Part { void** p; size_t bytes; };
  enkf::Workspace& ws = h.ws;
  Part parts[] = {
      // FP64 mode keeps HA and the solution in FP64; FP32 mode keeps them in double-float
      // only (HA64 and Z stay NULL, so the innovations kernel writes no FP64 HA)
      {(void**)&ws.HA64, fp64 ? 8 * mN : 0}, {(void**)&ws.D, 8 * mN}, {(void**)&ws.Z, fp64 ? 8 * mN : 0},
      {(void**)&ws.Res, vs * mN}, {(void**)&ws.P, vs * mN}, {(void**)&ws.Sv, vs * mN},
      {(void**)&ws.HA32, fp64 ? 0 : 4 * mN}, {(void**)&ws.B, fp64 ? 0 : vs * mN},
      {(void**)&ws.X, fp64 ? 0 : vs * mN}, {(void**)&ws.r32, fp64 ? 0 : 4 * size_t(c.m)},
      {(void**)&ws.HAdf, fp64 ? 0 : 8 * mN}, {(void**)&ws.Ddf, fp64 ? 0 : 8 * mN},
      {(void**)&ws.Zdf, fp64 ? 0 : 8 * mN},
      {(void**)&ws.Tpart, 8 * size_t(h.launch.G) * NE}, {(void**)&ws.Tred, 8 * NE},
      {(void**)&ws.rrpart, 8 * 2 * size_t(h.launch.G) * h.launch.NT},
      {(void**)&ws.Wacc, 8 * size_t(c.N) * c.N}, {(void**)&ws.W, 8 * size_t(c.N) * c.N},
      {(void**)&ws.col_iters, 4 * size_t(c.N)}, {(void**)&ws.col_relres, 8 * size_t(c.N)},
      {(void**)&ws.col_true, 8 * size_t(c.N)}, {(void**)&ws.status, 16}, {(void**)&ws.bar, 16},
  };
  size_t need = 0;
  for (const Part& q : parts) need += align256(q.bytes);
  if (need > kScratchBytes)   // too large for the fixed array: enkf_create serves it
    return noalloc_fail(ENKF_ERR_UNSUPPORTED, "enkf_analyze_noalloc: working memory exceeds the fixed array");
  void* base = nullptr;
  e = scratch_address(h.device, &base);
  if (e != cudaSuccess) return noalloc_fail(ENKF_ERR_CUDA, "enkf_analyze_noalloc: cudaGetSymbolAddress");
  size_t off = 0;
  for (const Part& q : parts) {
    *q.p = q.bytes ? static_cast<unsigned char*>(base) + off : nullptr;
    off += align256(q.bytes);
  }
  ws.rowptr = const_cast<int32_t*>(d_rowptr);
  ws.col = const_cast<int32_t*>(d_col);
  ws.w = const_cast<double*>(d_w);
  ws.r = const_cast<double*>(d_r);

  // launch_solve clears the barrier counter and status words before the solve; everything
  // else in the array is fully written before it is read within one call.
  if (!fp64) e = enkf::launch_convert_r(&h);
  if (e == cudaSuccess)
    e = enkf::launch_innovations(&h, d_Xf, d_y, nullptr, c.perturb_obs ? 2 : 0, seed, counter);
  if (e == cudaSuccess) e = enkf::launch_solve(&h);
  if (e == cudaSuccess) e = enkf::launch_update(&h, d_Xf, d_Xa);
  if (e != cudaSuccess) return noalloc_fail(ENKF_ERR_CUDA, "enkf_analyze_noalloc: launch");
  if (!out_stats) return ENKF_OK;

  // optional outcome: synchronise and fold the per-column results (host stack arrays only)
  int32_t it[128], st[4];
  double rel[128], tr[128];
  e = cudaStreamSynchronize(h.stream);
  if (e == cudaSuccess) e = cudaMemcpy(it, ws.col_iters, 4 * c.N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(rel, ws.col_relres, 8 * c.N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(tr, ws.col_true, 8 * c.N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(st, ws.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return noalloc_fail(ENKF_ERR_CUDA, "enkf_analyze_noalloc: stats");
  std::memset(out_stats, 0, sizeof(*out_stats));
  out_stats->iters_min = 1 << 30;
  out_stats->true_relres_max = -1.0;
  int conv = 0;
  for (int j = 0; j < c.N; ++j) {
    out_stats->iters_max = it[j] > out_stats->iters_max ? it[j] : out_stats->iters_max;
    out_stats->iters_min = it[j] < out_stats->iters_min ? it[j] : out_stats->iters_min;
    out_stats->relres_max = rel[j] > out_stats->relres_max ? rel[j] : out_stats->relres_max;
    if (tr[j] >= 0.0 && tr[j] > out_stats->true_relres_max) out_stats->true_relres_max = tr[j];
    conv += (c.fixed_iters > 0 || rel[j] <= c.tol) ? 1 : 0;
  }
  out_stats->refinements = st[1];
  out_stats->columns_converged = conv;
  out_stats->grid_blocks = h.launch.G;
  out_stats->warm_relres_max = -1.0;
  out_stats->warm_fallbacks = 0.0;
  enkf_status s = ENKF_OK;
  if (st[0] & enkf::DS_SMEM) s = ENKF_ERR_CUDA;
  else if (st[0] & enkf::DS_TIMEOUT) s = ENKF_ERR_TIMEOUT;
  else if (st[0] & enkf::DS_NONFINITE) s = ENKF_ERR_NONFINITE;
  else if (st[0] & enkf::DS_BREAKDOWN) s = ENKF_ERR_BREAKDOWN;
  else if (st[0] & enkf::DS_NOT_CONVERGED) s = ENKF_ERR_NOT_CONVERGED;
  out_stats->status = s;
  return s;
}

}  // extern "C"
