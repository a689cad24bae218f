// C ABI of libenkf.so (declared in include/enkf.h): argument checking, workspace
// ownership, and the enqueue order of one analysis step.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "intermediates.cuh"
#include "gram_stages.cuh"

using enkf::Workspace;

namespace {

thread_local std::string g_create_error;

enkf_status fail(enkf_handle_s* h, enkf_status s, const std::string& msg) {
  if (h) h->last_error = msg;
  else g_create_error = msg;
  return s;
}

enkf_status cuda_fail(enkf_handle_s* h, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? ENKF_ERR_OOM : ENKF_ERR_CUDA, msg);
}

void free_workspace(Workspace& ws) {
  void* ptrs[] = {ws.rowptr, ws.col, ws.w, ws.r, ws.r32, ws.HA64, ws.HA32, ws.HA16, ws.HAdf, ws.Ddf, ws.Zdf, ws.D, ws.Z, ws.B, ws.X,
                  ws.Res, ws.P, ws.Sv, ws.prof, ws.Tpart, ws.Tred, ws.rrpart, ws.Wacc, ws.W, ws.col_iters,
                  ws.col_relres, ws.col_true, ws.col_warm, ws.status, ws.bar, ws.stage_Xf, ws.stage_y,
                  ws.Hrowptr, ws.Hcol, ws.Hw, ws.wa, ws.wb, ws.wcp, ws.wmu, ws.wU, ws.wV, ws.wcarry,
                  ws.wcarryV, ws.Xw, ws.yw, ws.Tk, ws.Tacc, ws.hamax};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  ws = Workspace{};
}

// Argument checks shared by enkf_create and enkf_batch_create; on failure the message is
// left in msg (without the caller's prefix).
enkf_status check_problem(const enkf_config& c, const int32_t* h_rowptr, const int32_t* h_col,
                          const double* h_w, const double* r_diag, std::string& msg) {
  auto bad = [&](enkf_status s, const char* m) { msg = m; return s; };
  if (!h_rowptr || !r_diag) return bad(ENKF_ERR_INVALID_ARG, "NULL rowptr or r");
  if (c.n < 1 || c.m < 1 || c.N < 2)
    return bad(ENKF_ERR_INVALID_ARG, "need n >= 1, m >= 1, N >= 2");
  if (c.m >= (int64_t(1) << 32) || c.n >= (int64_t(1) << 31))
    return bad(ENKF_ERR_INVALID_ARG, "m must be < 2^32 and n < 2^31");
  if (c.N > 128) return bad(ENKF_ERR_UNSUPPORTED, "N > 128");
  if (c.precision < ENKF_FP64 || c.precision > ENKF_FP16_REFINE)
    return bad(ENKF_ERR_UNSUPPORTED, "unknown precision mode");
  const bool mixed = c.precision == ENKF_BF16_REFINE || c.precision == ENKF_FP16_REFINE;
  if (mixed && c.variant != ENKF_CGD)
    return bad(ENKF_ERR_UNSUPPORTED, "the BF16/FP16 modes are built for ENKF_CGD");
  if (mixed && c.fixed_iters > 0)
    return bad(ENKF_ERR_UNSUPPORTED, "fixed_iters is not offered in the BF16/FP16 modes");
  if (c.variant != ENKF_CGD && c.variant != ENKF_CGD_REDUCED && c.variant != ENKF_SENKF)
    return bad(ENKF_ERR_UNSUPPORTED, "unknown variant");
  if (c.fixed_iters < 0 || c.max_iter < 1 || c.max_refine < 0)
    return bad(ENKF_ERR_INVALID_ARG, "bad iteration limits");
  if (c.fixed_iters == 0 && !(c.tol > 0.0 && std::isfinite(c.tol)))
    return bad(ENKF_ERR_INVALID_ARG, "tol must be positive and finite");
  if (c.precision == ENKF_FP32 && !(c.inner_tol > 0.0 && c.inner_tol < 1.0))
    return bad(ENKF_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
  if (c.grid_blocks < 0) return bad(ENKF_ERR_INVALID_ARG, "grid_blocks < 0");
  if (c.precondition != 0 && c.precondition != 1)
    return bad(ENKF_ERR_INVALID_ARG, "precondition must be 0 or 1");
  if (c.lowprec_terms != 0 && c.lowprec_terms != 1 && c.lowprec_terms != 3)
    return bad(ENKF_ERR_INVALID_ARG, "lowprec_terms must be 0, 1 or 3");
  if (c.warm_start != 0 && c.warm_start != 1) return bad(ENKF_ERR_INVALID_ARG, "warm_start must be 0 or 1");
  if (c.warm_start && (c.precision != ENKF_FP32 || c.variant != ENKF_CGD || c.fixed_iters > 0))
    return bad(ENKF_ERR_UNSUPPORTED, "the learned warm start runs in ENKF_CGD / ENKF_FP32 without fixed_iters");
  if (c.warm_accept != 0 && c.warm_accept != 1) return bad(ENKF_ERR_INVALID_ARG, "warm_accept must be 0 or 1");
  if (c.reduce_order != 0 && c.reduce_order != 1) return bad(ENKF_ERR_INVALID_ARG, "reduce_order must be 0 or 1");
  for (int q = 0; q < 3; ++q)
    if (c.reserved[q]) return bad(ENKF_ERR_INVALID_ARG, "reserved fields must be 0");
  // observation operator and R
  if (h_rowptr[0] != 0) return bad(ENKF_ERR_INVALID_ARG, "rowptr[0] != 0");
  for (int64_t i = 0; i < c.m; ++i)
    if (h_rowptr[i + 1] < h_rowptr[i])
      return bad(ENKF_ERR_INVALID_ARG, "rowptr decreases");
  const int64_t nnz = h_rowptr[c.m];
  if (nnz > 0 && (!h_col || !h_w))
    return bad(ENKF_ERR_INVALID_ARG, "NULL col/w with nnz > 0");
  for (int64_t k = 0; k < nnz; ++k) {
    if (h_col[k] < 0 || h_col[k] >= c.n)
      return bad(ENKF_ERR_INVALID_ARG, "column index outside [0, n)");
    if (!std::isfinite(h_w[k])) return bad(ENKF_ERR_INVALID_ARG, "non-finite weight");
  }
  for (int64_t i = 0; i < c.m; ++i)
    if (!(r_diag[i] > 0.0) || !std::isfinite(r_diag[i]))
      return bad(ENKF_ERR_INVALID_ARG, "r must be positive and finite");

  return ENKF_OK;
}

size_t elem_size(const enkf_config& c) { return c.precision == ENKF_FP64 ? 8 : 4; }

}  // namespace

extern "C" {

enkf_status enkf_config_default(enkf_config* cfg, int64_t n, int64_t m, int32_t N) {
  if (!cfg) return ENKF_ERR_INVALID_ARG;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->n = n;
  cfg->m = m;
  cfg->N = N;
  cfg->precision = ENKF_FP64;
  cfg->variant = ENKF_CGD;
  cfg->max_iter = 1000;
  cfg->tol = 1e-8;
  cfg->fixed_iters = 0;
  cfg->max_refine = 4;
  cfg->inner_tol = 1e-5;
  cfg->refresh_every = 0;
  cfg->perturb_obs = 1;
  cfg->warm_start = 0;
  cfg->true_residual = 1;
  cfg->grid_blocks = 0;
  return ENKF_OK;
}

const char* enkf_status_str(enkf_status s) {
  switch (s) {
    case ENKF_OK: return "ok";
    case ENKF_ERR_INVALID_ARG: return "invalid argument";
    case ENKF_ERR_CUDA: return "CUDA error";
    case ENKF_ERR_OOM: return "out of device memory";
    case ENKF_ERR_NOT_CONVERGED: return "CG did not converge within max_iter";
    case ENKF_ERR_NONFINITE: return "non-finite value in the inputs or the CG recurrences";
    case ENKF_ERR_BREAKDOWN: return "CG breakdown (p^T S p <= 0)";
    case ENKF_ERR_TIMEOUT: return "device grid barrier timed out";
    case ENKF_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

const char* enkf_last_error(enkf_handle h) {
  return h ? h->last_error.c_str() : g_create_error.c_str();
}

static enkf_status create_impl(const enkf_config* cfg, const int32_t* h_rowptr, const int32_t* h_col,
                               const double* h_w, const double* r_diag, const double* r_off,
                               void* cuda_stream, enkf_handle* out) {
  if (out) *out = nullptr;
  if (!cfg || !out || !h_rowptr || !r_diag)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_create: NULL argument");
  const enkf_config c = *cfg;
  {
    std::string msg;
    const enkf_status cs = check_problem(c, h_rowptr, h_col, h_w, r_diag, msg);
    if (cs != ENKF_OK) return fail(nullptr, cs, "enkf_create: " + msg);
  }
  // tridiagonal R: the sEnKF comparator uses only the diagonal of R (Algorithm 3); the other
  // forms analyse the whitened problem (kernels_whiten.cu)
  const bool tri = r_off != nullptr && c.variant != ENKF_SENKF && c.m > 1;
  std::vector<double> wa, wb, wcp, wmu;
  if (tri) {
    for (int64_t i = 0; i + 1 < c.m; ++i)
      if (!std::isfinite(r_off[i])) return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_create: non-finite r_off");
    if (c.variant == ENKF_CGD && c.precondition != 1)
      return fail(nullptr, ENKF_ERR_UNSUPPORTED,
                  "enkf_create: a tridiagonal R needs precondition = 1 in ENKF_CGD (CG preconditioned by R)");
    if (!enkf::whiten_coefficients(c.m, r_diag, r_off, wa, wb, wcp, wmu))
      return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_create: R is not positive definite");
  }
  const bool mixed = c.precision == ENKF_BF16_REFINE || c.precision == ENKF_FP16_REFINE;
  const int64_t nnz = tri ? c.m : h_rowptr[c.m];
  auto* h = new enkf_handle_s();
  h->cfg = c;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->nnz = nnz;
  h->tri = tri;
  if (!tri && c.m > 0) {
    double sl = 0.0;
    for (int64_t i = 0; i < c.m; ++i) sl += std::log2(r_diag[i]);
    const long k = std::lround(sl / (double)c.m);
    h->r_pow2 = std::ldexp(1.f, (int)std::max(-120L, std::min(120L, k)));
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = mixed ? enkf::plan_solve_mixed(h) : enkf::plan_solve(h);
  if (e != cudaSuccess) {
    enkf_status s = cuda_fail(nullptr, e, "enkf_create: device query / planning");
    delete h;
    return s;
  }
  const int64_t mN = c.m * c.N;
  const int G = h->launch.G, NT = h->launch.NT;
  const int64_t NE = (int64_t)c.N * c.N + 4 * c.N;   // partials: N x N Gram + four column-sum vectors
  const size_t vs = elem_size(c);
  Workspace& ws = h->ws;
  struct Alloc { void** p; size_t bytes; };
  // the Reduced variant and the sEnKF comparator work from one Gram pass and keep no m x N arrays
  const bool gram = c.variant != ENKF_CGD;
  const int64_t tpart = gram ? (int64_t)enkf::reduced_grid(h) * 2 * c.N * c.N : (int64_t)G * NE;
  std::vector<Alloc> allocs = {
      {(void**)&ws.rowptr, sizeof(int32_t) * (c.m + 1)},
      {(void**)&ws.col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)},
      {(void**)&ws.w, sizeof(double) * (size_t)std::max<int64_t>(nnz, 1)},
      {(void**)&ws.r, sizeof(double) * c.m},
      {(void**)&ws.Tpart, sizeof(double) * tpart},
      {(void**)&ws.Tred, sizeof(double) * NE},
      {(void**)&ws.rrpart, sizeof(double) * 2 * G * NT},
      {(void**)&ws.Wacc, sizeof(double) * c.N * c.N},
      {(void**)&ws.W, sizeof(double) * c.N * c.N},
      {(void**)&ws.col_iters, sizeof(int32_t) * c.N},
      {(void**)&ws.col_relres, sizeof(double) * c.N},
      {(void**)&ws.col_true, sizeof(double) * c.N},
      {(void**)&ws.col_warm, sizeof(double) * c.N},
      {(void**)&ws.status, sizeof(int32_t) * 4},
      {(void**)&ws.bar, sizeof(unsigned) * 4},
      {(void**)&ws.stage_Xf, vs * c.n * c.N},
      {(void**)&ws.stage_y, sizeof(double) * c.m},
      {(void**)&ws.prof, sizeof(unsigned long long) * 8},
  };
  if (!gram) {
    allocs.push_back({(void**)&ws.Sv, vs * mN});
    allocs.push_back({(void**)&ws.D, sizeof(double) * mN});
    allocs.push_back({(void**)&ws.Res, vs * mN});
    allocs.push_back({(void**)&ws.P, vs * mN});
    if (c.precision == ENKF_FP64) {   // the other modes keep HA and Z in double-float only
      allocs.push_back({(void**)&ws.HA64, sizeof(double) * mN});
      allocs.push_back({(void**)&ws.Z, sizeof(double) * mN});
    }
  }
  if (!gram && c.precision != ENKF_FP64) {
    allocs.push_back({(void**)&ws.HA32, sizeof(float) * mN});
    allocs.push_back({(void**)&ws.r32, sizeof(float) * c.m});
    allocs.push_back({(void**)&ws.B, vs * mN});
    allocs.push_back({(void**)&ws.X, vs * mN});
    allocs.push_back({(void**)&ws.HAdf, 8 * (size_t)mN});
    allocs.push_back({(void**)&ws.Ddf, 8 * (size_t)mN});
    allocs.push_back({(void**)&ws.Zdf, 8 * (size_t)mN});
  }
  if (mixed) {
    allocs.push_back({(void**)&ws.HA16, enkf::mixed_image_bytes(h)});
    allocs.push_back({(void**)&ws.Tk, sizeof(float) * 2 * c.N * c.N});
    allocs.push_back({(void**)&ws.hamax, sizeof(unsigned) * 4});
  }
  if (c.precision != ENKF_FP64 && c.variant == ENKF_CGD)
    allocs.push_back({(void**)&ws.Tacc, sizeof(double) * 3 * ((size_t)c.N * c.N + 4 * c.N)});
  const int64_t hnnz = h_rowptr[c.m];
  const int64_t nblk = enkf::whiten_blocks(c.m);
  if (tri) {
    allocs.push_back({(void**)&ws.Hrowptr, sizeof(int32_t) * (c.m + 1)});
    allocs.push_back({(void**)&ws.Hcol, sizeof(int32_t) * (size_t)std::max<int64_t>(hnnz, 1)});
    allocs.push_back({(void**)&ws.Hw, sizeof(double) * (size_t)std::max<int64_t>(hnnz, 1)});
    allocs.push_back({(void**)&ws.wa, sizeof(double) * c.m});
    allocs.push_back({(void**)&ws.wb, sizeof(double) * c.m});
    allocs.push_back({(void**)&ws.wcp, sizeof(double) * c.m});
    allocs.push_back({(void**)&ws.wmu, sizeof(double) * nblk});
    allocs.push_back({(void**)&ws.wU, sizeof(double) * c.m * (c.N + 1)});
    allocs.push_back({(void**)&ws.wV, sizeof(double) * mN});
    allocs.push_back({(void**)&ws.wcarry, sizeof(double) * nblk * (c.N + 1)});
    allocs.push_back({(void**)&ws.wcarryV, sizeof(double) * nblk * c.N});
    allocs.push_back({(void**)&ws.Xw, vs * mN});
    allocs.push_back({(void**)&ws.yw, sizeof(double) * c.m});
  }
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      free_workspace(ws);
      delete h;
      return cuda_fail(nullptr, e, "enkf_create: cudaMalloc");
    }
  }
  if (!tri) {
    e = cudaMemcpy(ws.rowptr, h_rowptr, sizeof(int32_t) * (c.m + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(ws.col, h_col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(ws.w, h_w, sizeof(double) * nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.r, r_diag, sizeof(double) * c.m, cudaMemcpyHostToDevice);
  } else {
    // the whitened problem: H' = I, r' = 1; the caller's H for the whitening pass
    std::vector<int32_t> idx(c.m + 1);
    for (int64_t i = 0; i <= c.m; ++i) idx[i] = (int32_t)i;
    const std::vector<double> ones(c.m, 1.0);
    e = cudaMemcpy(ws.rowptr, idx.data(), sizeof(int32_t) * (c.m + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.col, idx.data(), sizeof(int32_t) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.w, ones.data(), sizeof(double) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.r, ones.data(), sizeof(double) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.Hrowptr, h_rowptr, sizeof(int32_t) * (c.m + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && hnnz > 0) e = cudaMemcpy(ws.Hcol, h_col, sizeof(int32_t) * hnnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && hnnz > 0) e = cudaMemcpy(ws.Hw, h_w, sizeof(double) * hnnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.wa, wa.data(), sizeof(double) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.wb, wb.data(), sizeof(double) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.wcp, wcp.data(), sizeof(double) * c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ws.wmu, wmu.data(), sizeof(double) * nblk, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(ws.status, 0, sizeof(int32_t) * 4);
  if (e == cudaSuccess && ws.HA16) e = cudaMemset(ws.HA16, 0, enkf::mixed_image_bytes(h));
  if (e == cudaSuccess) e = cudaMemset(ws.bar, 0, sizeof(unsigned) * 4);
  if (e == cudaSuccess) e = enkf::launch_convert_r(h);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    free_workspace(ws);
    delete h;
    return cuda_fail(nullptr, e, "enkf_create: upload");
  }
  *out = h;
  return ENKF_OK;
}

enkf_status enkf_create(const enkf_config* cfg, const int32_t* h_rowptr, const int32_t* h_col,
                        const double* h_w, const double* r_diag, void* cuda_stream,
                        enkf_handle* out) {
  return create_impl(cfg, h_rowptr, h_col, h_w, r_diag, nullptr, cuda_stream, out);
}

enkf_status enkf_create_tridiag(const enkf_config* cfg, const int32_t* h_rowptr, const int32_t* h_col,
                                const double* h_w, const double* r_diag, const double* r_off,
                                void* cuda_stream, enkf_handle* out) {
  if (cfg && cfg->m > 1 && !r_off)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_create_tridiag: NULL r_off");
  return create_impl(cfg, h_rowptr, h_col, h_w, r_diag, r_off, cuda_stream, out);
}

// An upload of X_f that runs on the handle's copy stream once the innovations are done (their
// reads of host memory then have the CPU-GPU link to themselves) and that the update waits for.
struct XfUpload {
  void* dst;
  const void* src;
  size_t bytes;
};

// d_Xf feeds the innovations (the observed rows of X_f); the update reads d_Xf_upd (nullptr:
// d_Xf), after the upload `up` (if given) has completed.
static enkf_status analyze_impl(enkf_handle h, const void* d_Xf, const double* d_y,
                                const double* d_E, int emode, uint64_t seed, uint64_t counter,
                                void* d_Xa, const void* d_Xf_upd = nullptr, const XfUpload* up = nullptr) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "analyze: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "analyze: batched handle (use the enkf_batch_* calls)");
  if (!d_Xf || !d_y || !d_Xa) return fail(h, ENKF_ERR_INVALID_ARG, "analyze: NULL X_f, y or X_a");
  const auto& c = h->cfg;
  const size_t xb = elem_size(c) * c.n * c.N;
  if (!d_Xf_upd) d_Xf_upd = d_Xf;
  const char* a = static_cast<const char*>(d_Xf_upd);
  const char* b = static_cast<const char*>(d_Xa);
  if (a != b && a < b + xb && b < a + xb)
    return fail(h, ENKF_ERR_INVALID_ARG, "analyze: X_a partially overlaps X_f");
  cudaError_t e = cudaSuccess;
  // Reduced and sEnKF: a Gram pass over the observation rows, then an N x N stage (both
  // variants form HA and D inside the Gram pass instead of the innovations kernel)
  const bool gram = c.variant != ENKF_CGD;
  if (h->timing) e = cudaEventRecord(h->ev[0], h->stream);
  if (c.warm_start && !enkf::warm_ready(h))
    return fail(h, ENKF_ERR_INVALID_ARG, "analyze: warm_start = 1 but no model attached (enkf_set_warm_model)");
  // tridiagonal R: the observation rows are whitened first and the analysis runs on the
  // whitened problem (H' = I, r' = 1); the update below still uses the caller's X_f
  const void* Xin = d_Xf;
  const double* yin = d_y;
  const double* Ein = d_E;
  if (h->tri && e == cudaSuccess) {
    e = enkf::launch_whiten(h, d_Xf, d_y, emode == 1 ? d_E : nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze: whitening launch");
    Xin = h->ws.Xw;
    yin = h->ws.yw;
    Ein = emode == 1 ? h->ws.wV : nullptr;
  }
  if (e == cudaSuccess)
    e = gram ? enkf::launch_gram_stage(h, Xin, yin, Ein, emode, seed, counter)
             : enkf::launch_innovations(h, Xin, yin, Ein, emode, seed, counter);
  if (e != cudaSuccess) return cuda_fail(h, e, gram ? "analyze: Gram pass launch" : "analyze: innovations launch");
  if (up) {
    e = cudaEventRecord(h->host_ev[0], h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->host_ev[0], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(up->dst, up->src, up->bytes, cudaMemcpyHostToDevice, h->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->host_ev[1], h->copy_stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze: upload of X_f");
  }
  if (c.warm_start) {
    e = enkf::warm_prepare(h);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze: learned warm start");
  }
  if (h->timing) e = cudaEventRecord(h->ev[1], h->stream);
  if (e == cudaSuccess)
    e = gram ? enkf::launch_nxn_stage(h)
             : (h->cfg.precision >= ENKF_BF16_REFINE ? enkf::launch_solve_mixed(h) : enkf::launch_solve(h));
  if (e != cudaSuccess) return cuda_fail(h, e, "analyze: CG launch");
  if (h->timing) e = cudaEventRecord(h->ev[2], h->stream);
  if (e == cudaSuccess && up) e = cudaStreamWaitEvent(h->stream, h->host_ev[1], 0);
  if (e == cudaSuccess)
    e = c.variant == ENKF_CGD_REDUCED ? enkf::launch_update_product(h, d_Xf_upd, d_Xa)
                                      : enkf::launch_update(h, d_Xf_upd, d_Xa);
  if (e != cudaSuccess) return cuda_fail(h, e, "analyze: update launch");
  if (h->timing) {
    e = cudaEventRecord(h->ev[3], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze: timing event");
    h->timed = true;
  }
  h->has_result = true;
  return ENKF_OK;
}

enkf_status enkf_analyze(enkf_handle h, const void* d_Xf, const double* d_y, uint64_t seed,
                         uint64_t counter, void* d_Xa) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "analyze: NULL handle");
  return analyze_impl(h, d_Xf, d_y, nullptr, h->cfg.perturb_obs ? 2 : 0, seed, counter, d_Xa);
}

enkf_status enkf_analyze_with_E(enkf_handle h, const void* d_Xf, const double* d_y,
                                const double* d_E, void* d_Xa) {
  return analyze_impl(h, d_Xf, d_y, d_E, d_E ? 1 : 0, 0, 0, d_Xa);
}

// The device address of pinned (page-locked, mapped) host memory, or nullptr for any other
// pointer (pageable host memory, device memory).
static void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // clear the error of an unknown pointer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

enkf_status enkf_analyze_host(enkf_handle h, const void* h_Xf, const double* h_y, uint64_t seed,
                              uint64_t counter, void* h_Xa) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "analyze_host: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "analyze_host: batched handle (use the enkf_batch_* calls)");
  if (!h_Xf || !h_y || !h_Xa) return fail(h, ENKF_ERR_INVALID_ARG, "analyze_host: NULL buffer");
  const auto& c = h->cfg;
  const size_t xb = elem_size(c) * c.n * c.N;
  const void* xf_dev = device_view(h_Xf);
  void* xa_dev = device_view(h_Xa);
  if (xf_dev && c.variant == ENKF_CGD) {
    // Pinned X_f: the innovations read the observed rows of X_f directly from host memory (over
    // the CPU-GPU link); the whole X_f is then uploaded on the copy stream while the solve runs,
    // and only the update waits for it. A pinned X_a is written by the update kernel itself
    // (its coalesced 16-byte stores reach host memory about as fast as a copy does, and the
    // separate download disappears); otherwise X_a goes back by one copy.
    cudaError_t e = cudaSuccess;
    if (!h->copy_stream) {
      e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
      for (auto& ev : h->host_ev)
        if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e != cudaSuccess) return cuda_fail(h, e, "analyze_host: copy stream");
    }
    // (the upload starts after the innovations: run concurrently with them, it slowed their
    // reads of host memory from 0.14 to 0.25 ms at n = 262,144, N = 64)
    e = cudaMemcpyAsync(h->ws.stage_y, h_y, sizeof(double) * c.m, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze_host: upload");
    const XfUpload up{h->ws.stage_Xf, h_Xf, xb};
    enkf_status s = analyze_impl(h, xf_dev, h->ws.stage_y, nullptr, h->cfg.perturb_obs ? 2 : 0, seed, counter,
                                 xa_dev ? xa_dev : h->ws.stage_Xf, h->ws.stage_Xf, &up);
    if (s != ENKF_OK) {
      cudaStreamSynchronize(h->copy_stream);
      return s;
    }
    if (!xa_dev) e = cudaMemcpyAsync(h_Xa, h->ws.stage_Xf, xb, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "analyze_host: download");
    return ENKF_OK;
  }
  cudaError_t e = cudaMemcpyAsync(h->ws.stage_Xf, h_Xf, xb, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws.stage_y, h_y, sizeof(double) * c.m, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "analyze_host: upload");
  enkf_status s = enkf_analyze(h, h->ws.stage_Xf, h->ws.stage_y, seed, counter, h->ws.stage_Xf);
  if (s != ENKF_OK) return s;
  e = cudaMemcpyAsync(h_Xa, h->ws.stage_Xf, xb, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "analyze_host: download");
  return ENKF_OK;
}

enkf_status enkf_get_column_stats(enkf_handle h, int32_t* iters, double* relres, double* true_relres) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "get_column_stats: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "get_column_stats: batched handle (use the enkf_batch_* calls)");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  const int N = h->cfg.N;
  if (e == cudaSuccess && iters) e = cudaMemcpy(iters, h->ws.col_iters, sizeof(int32_t) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && relres) e = cudaMemcpy(relres, h->ws.col_relres, sizeof(double) * N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && true_relres) e = cudaMemcpy(true_relres, h->ws.col_true, sizeof(double) * N, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_column_stats");
  return ENKF_OK;
}

enkf_status enkf_get_stats(enkf_handle h, enkf_stats* out) {
  if (!h || !out) return fail(h, ENKF_ERR_INVALID_ARG, "get_stats: NULL argument");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "get_stats: batched handle (use enkf_batch_get_stats)");
  std::memset(out, 0, sizeof(*out));
  const int N = h->cfg.N;
  std::vector<int32_t> it(N);
  std::vector<double> rel(N), tr(N);
  enkf_status s = enkf_get_column_stats(h, it.data(), rel.data(), tr.data());
  if (s != ENKF_OK) return s;
  int32_t st[4];
  cudaError_t e = cudaMemcpy(st, h->ws.status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_stats");
  out->iters_max = 0;
  out->iters_min = 1 << 30;
  out->relres_max = 0.0;
  out->true_relres_max = -1.0;
  for (int j = 0; j < N; ++j) {
    out->iters_max = std::max(out->iters_max, it[j]);
    out->iters_min = std::min(out->iters_min, it[j]);
    out->relres_max = std::max(out->relres_max, rel[j]);
    if (tr[j] >= 0.0) out->true_relres_max = std::max(out->true_relres_max, tr[j]);
  }
  const int bits = st[0];
  out->refinements = st[1];
  out->warm_relres_max = -1.0;
  out->warm_fallbacks = 0.0;
  if (h->cfg.warm_start) {
    std::vector<double> wr(N);
    e = cudaMemcpy(wr.data(), h->ws.col_warm, sizeof(double) * N, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_stats");
    for (int j = 0; j < N; ++j) out->warm_relres_max = std::max(out->warm_relres_max, wr[j]);
    out->warm_fallbacks = st[2];
  }
  out->grid_blocks = h->launch.G;
  enkf_status status = ENKF_OK;
  if (bits & enkf::DS_SMEM) status = ENKF_ERR_CUDA;
  else if (bits & enkf::DS_TIMEOUT) status = ENKF_ERR_TIMEOUT;
  else if (bits & enkf::DS_NONFINITE) status = ENKF_ERR_NONFINITE;
  else if (bits & enkf::DS_BREAKDOWN) status = ENKF_ERR_BREAKDOWN;
  else if (bits & enkf::DS_NOT_CONVERGED) status = ENKF_ERR_NOT_CONVERGED;
  int conv = 0;
  const double tol = h->cfg.tol;
  for (int j = 0; j < N; ++j) conv += (h->cfg.fixed_iters > 0 || rel[j] <= tol) ? 1 : 0;
  out->columns_converged = conv;
  out->status = status;
  return status;
}

enkf_status enkf_copy_intermediates(enkf_handle h, double* d_HA, double* d_D, double* d_Z, double* d_W) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "copy_intermediates: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "copy_intermediates: batched handle (use the enkf_batch_* calls)");
  const auto& c = h->cfg;
  const size_t mN = sizeof(double) * c.m * c.N;
  cudaError_t e = cudaSuccess;
  if (c.variant == ENKF_SENKF) {
    if (d_HA || d_D || d_Z)
      return fail(h, ENKF_ERR_INVALID_ARG, "copy_intermediates: the sEnKF variant keeps no HA, D or Z");
    if (d_W) e = cudaMemcpyAsync(d_W, h->ws.W, sizeof(double) * c.N * c.N, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy_intermediates");
    return ENKF_OK;
  }
  if (c.variant == ENKF_CGD_REDUCED) {
    if (d_HA || d_D) return fail(h, ENKF_ERR_INVALID_ARG, "copy_intermediates: the reduced variant keeps no HA or D");
    const size_t nn = sizeof(double) * c.N * c.N;
    if (d_Z) e = cudaMemcpyAsync(d_Z, h->ws.W, nn, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && d_W) e = cudaMemcpyAsync(d_W, h->ws.Tred, nn, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "copy_intermediates");
    return ENKF_OK;
  }
  if (c.precision == ENKF_FP64) {
    if (d_HA) e = cudaMemcpyAsync(d_HA, h->ws.HA64, mN, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && d_Z) e = cudaMemcpyAsync(d_Z, h->ws.Z, mN, cudaMemcpyDeviceToDevice, h->stream);
  } else {   // HA and the solution Z live in double-float (FP32 pairs) in these modes
    const int64_t cnt = c.m * c.N;
    if (d_HA) e = enkf::launch_df32_to_f64(h->ws.HAdf, d_HA, cnt, h->stream);
    if (e == cudaSuccess && d_Z) e = enkf::launch_df32_to_f64(h->ws.Zdf, d_Z, cnt, h->stream);
  }
  if (e == cudaSuccess && d_D) e = cudaMemcpyAsync(d_D, h->ws.D, mN, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && d_W)
    e = cudaMemcpyAsync(d_W, h->ws.W, sizeof(double) * c.N * c.N, cudaMemcpyDeviceToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "copy_intermediates");
  return ENKF_OK;
}

enkf_status enkf_draw_perturbations(uint64_t seed, uint64_t counter, const double* d_r, int64_t m,
                                    int32_t N, double* d_E, void* cuda_stream) {
  if (!d_r || !d_E || m < 1 || N < 1)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "draw_perturbations: bad argument");
  cudaError_t e = enkf::launch_draw_perturbations(seed, counter, d_r, m, N, d_E,
                                                  static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "draw_perturbations");
  return ENKF_OK;
}

enkf_status enkf_set_phase_timing(enkf_handle h, int32_t enable) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "set_phase_timing: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "set_phase_timing: batched handle (use the enkf_batch_* calls)");
  if (enable && !h->ev[0]) {
    for (auto& ev : h->ev) {
      cudaError_t e = cudaEventCreate(&ev);
      if (e != cudaSuccess) return cuda_fail(h, e, "set_phase_timing: cudaEventCreate");
    }
  }
  h->timing = enable != 0;
  h->prof_enabled = enable >= 2;
  h->timed = false;
  return ENKF_OK;
}

enkf_status enkf_get_solve_phases(enkf_handle h, double* us) {
  if (!h || !us) return fail(h, ENKF_ERR_INVALID_ARG, "get_solve_phases: NULL argument");
  if (!h->prof_enabled || !h->timed) return fail(h, ENKF_ERR_INVALID_ARG, "get_solve_phases: phase timers off");
  unsigned long long ns[8];
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(ns, h->ws.prof, sizeof(ns), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_solve_phases");
  for (int q = 0; q < 8; ++q) us[q] = 1e-3 * (double)ns[q];
  return ENKF_OK;
}

enkf_status enkf_get_phase_times(enkf_handle h, float* ms) {
  if (!h || !ms) return fail(h, ENKF_ERR_INVALID_ARG, "get_phase_times: NULL argument");
  if (!h->timing || !h->timed) return fail(h, ENKF_ERR_INVALID_ARG, "get_phase_times: no timed analysis");
  cudaError_t e = cudaEventSynchronize(h->ev[3]);
  for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaEventElapsedTime(&ms[q], h->ev[q], h->ev[q + 1]);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_phase_times");
  return ENKF_OK;
}

// ------------------------------------------------------------------ batched analyses
enkf_status enkf_batch_create(int32_t count, const enkf_config* cfgs,
                              const int32_t* const* h_rowptr, const int32_t* const* h_col,
                              const double* const* h_w, const double* const* r_diag,
                              void* cuda_stream, enkf_handle* out) {
  if (out) *out = nullptr;
  if (!cfgs || !out || !h_rowptr || !h_col || !h_w || !r_diag || count < 1)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_create: NULL argument or count < 1");
  for (int32_t i = 0; i < count; ++i) {
    const enkf_config& c = cfgs[i];
    std::string msg;
    const enkf_status cs = check_problem(c, h_rowptr[i], h_col[i], h_w[i], r_diag[i], msg);
    const std::string who = "enkf_batch_create: problem " + std::to_string(i) + ": ";
    if (cs != ENKF_OK) return fail(nullptr, cs, who + msg);
    if (c.precision != ENKF_FP32 || c.variant != ENKF_CGD || c.precondition != 1 || c.fixed_iters != 0)
      return fail(nullptr, ENKF_ERR_UNSUPPORTED,
                  who + "batches run ENKF_CGD in ENKF_FP32 with precondition = 1 and fixed_iters = 0");
    if (c.perturb_obs != cfgs[0].perturb_obs)
      return fail(nullptr, ENKF_ERR_INVALID_ARG, who + "perturb_obs differs from problem 0");
  }
  auto* h = new enkf_handle_s();
  h->cfg = cfgs[0];
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  std::string err = "enkf_batch_create: device query";
  if (e == cudaSuccess) e = enkf::batch_build(h, count, cfgs, h_rowptr, h_col, h_w, r_diag, err);
  if (e != cudaSuccess) {
    enkf_status s = cuda_fail(nullptr, e, err.c_str());
    enkf::batch_free(h);
  enkf::warm_free(h);
    delete h;
    return s;
  }
  *out = h;
  return ENKF_OK;
}

static enkf_status batch_args(enkf_handle h, const void* const* d_Xf, const double* const* d_y,
                              void* const* d_Xa, const char* who) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, std::string(who) + ": NULL handle");
  if (!h->batch) return fail(h, ENKF_ERR_INVALID_ARG, std::string(who) + ": not a batched handle");
  if (!d_Xf || !d_y || !d_Xa) return fail(h, ENKF_ERR_INVALID_ARG, std::string(who) + ": NULL pointer array");
  const int count = enkf::batch_count(h);
  for (int i = 0; i < count; ++i) {
    if (!d_Xf[i] || !d_y[i] || !d_Xa[i])
      return fail(h, ENKF_ERR_INVALID_ARG, std::string(who) + ": NULL X_f, y or X_a of problem " + std::to_string(i));
    const size_t xb = enkf::batch_state_bytes(h, i);
    const char* a = static_cast<const char*>(d_Xf[i]);
    const char* b = static_cast<const char*>(d_Xa[i]);
    if (a != b && a < b + xb && b < a + xb)
      return fail(h, ENKF_ERR_INVALID_ARG, std::string(who) + ": X_a partially overlaps X_f in problem " + std::to_string(i));
  }
  return ENKF_OK;
}

enkf_status enkf_batch_analyze(enkf_handle h, const void* const* d_Xf, const double* const* d_y,
                               const uint64_t* seeds, const uint64_t* counters, void* const* d_Xa) {
  enkf_status s = batch_args(h, d_Xf, d_y, d_Xa, "enkf_batch_analyze");
  if (s != ENKF_OK) return s;
  cudaError_t e = enkf::batch_analyze(h, d_Xf, d_y, seeds, counters, d_Xa);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_batch_analyze");
  h->has_result = true;
  return ENKF_OK;
}

enkf_status enkf_batch_tune(enkf_handle h, const void* const* d_Xf, const double* const* d_y,
                            const uint64_t* seeds, const uint64_t* counters, void* const* d_Xa,
                            double* best_ms) {
  enkf_status s = batch_args(h, d_Xf, d_y, d_Xa, "enkf_batch_tune");
  if (s != ENKF_OK) return s;
  double alpha = 0.0;
  cudaError_t e = enkf::batch_tune(h, d_Xf, d_y, seeds, counters, d_Xa, &alpha, best_ms);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_batch_tune");
  h->has_result = true;
  return ENKF_OK;
}

enkf_status enkf_batch_get_stats(enkf_handle h, int32_t* status, int32_t* iters_max,
                                 double* relres_max, int32_t* refinements) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_get_stats: NULL handle");
  if (!h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_stats: not a batched handle");
  if (!h->has_result) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_stats: no analysis yet");
  const int count = enkf::batch_count(h);
  std::vector<int32_t> st(count);
  cudaError_t e = enkf::batch_stats(h, st.data(), iters_max, relres_max, refinements);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_batch_get_stats");
  enkf_status worst = ENKF_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = st[i];
    if (worst == ENKF_OK && st[i] != ENKF_OK) worst = (enkf_status)st[i];
  }
  return worst;
}

enkf_status enkf_batch_get_plan(enkf_handle h, int32_t* grid, int32_t* teams, double* alpha,
                                int32_t* graphed) {
  if (!h || !h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_plan: not a batched handle");
  const enkf::BatchPlanOut p = enkf::batch_info(h);
  if (grid) *grid = p.grid;
  if (teams) *teams = p.teams;
  if (alpha) *alpha = p.alpha;
  if (graphed) *graphed = p.graphed;
  return ENKF_OK;
}

enkf_status enkf_batch_get_row_floors(enkf_handle h, int32_t* row_floors) {
  if (!h || !h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_row_floors: not a batched handle");
  if (!row_floors) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_row_floors: NULL output");
  const enkf::BatchPlanOut p = enkf::batch_info(h);
  for (int q = 0; q < 4; ++q) row_floors[q] = p.row_floors[q];
  return ENKF_OK;
}

enkf_status enkf_selftest_wait_timeout(int32_t which, double timeout_ms, void* cuda_stream) {
  if ((which != 0 && which != 1) || !(timeout_ms > 0.0 && timeout_ms <= 10000.0))
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_selftest_wait_timeout: which must be 0 or 1, timeout_ms in (0, 1e4]");
  int bits = 0;
  cudaError_t e = enkf::selftest_wait_timeout(which, timeout_ms, static_cast<cudaStream_t>(cuda_stream), &bits);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "enkf_selftest_wait_timeout");
  if (bits & enkf::DS_TIMEOUT) return ENKF_ERR_TIMEOUT;
  return fail(nullptr, ENKF_ERR_CUDA, "enkf_selftest_wait_timeout: the wait was not reported as timed out");
}

enkf_status enkf_batch_set_phase_timing(enkf_handle h, int32_t enable) {
  if (!h || !h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_set_phase_timing: not a batched handle");
  cudaError_t e = enkf::batch_set_phase_timing(h, enable != 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_batch_set_phase_timing");
  return ENKF_OK;
}

enkf_status enkf_batch_get_times(enkf_handle h, double* start_us, double* end_us, double* phase_us,
                                 int32_t* team_size) {
  if (!h || !h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_times: not a batched handle");
  if (!h->has_result) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_times: no analysis yet");
  if (phase_us && !enkf::batch_phase_timing(h))
    return fail(h, ENKF_ERR_INVALID_ARG, "enkf_batch_get_times: phase timers off (enkf_batch_set_phase_timing)");
  cudaError_t e = enkf::batch_times(h, start_us, end_us, phase_us, team_size);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_batch_get_times");
  return ENKF_OK;
}

enkf_status enkf_batch_plan(int32_t count, const enkf_config* cfgs, int32_t max_grid, double alpha,
                            const int32_t* row_floors, int32_t* cta_team, int32_t* cta_rank,
                            int32_t* team_size, int32_t* team_first, int32_t* order, int32_t* grid,
                            int32_t* teams) {
  if (count < 1 || !cfgs || max_grid < 1 || !(alpha > 0.0 && alpha <= 1.0))
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_plan: bad argument");
  if (row_floors)
    for (int q = 0; q < 4; ++q)
      if (row_floors[q] < 1) return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_plan: row floor < 1");
  for (int32_t i = 0; i < count; ++i)
    if (cfgs[i].m < 1 || cfgs[i].n < 1 || cfgs[i].N < 2 || cfgs[i].N > 128)
      return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_plan: bad problem shape");
  enkf::BatchPlanOut p;
  if (!enkf::batch_plan_host(count, cfgs, max_grid, alpha, row_floors, cta_team, cta_rank, team_size,
                             team_first, order, &p))
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_batch_plan: planning failed");
  if (grid) *grid = p.grid;
  if (teams) *teams = p.teams;
  return ENKF_OK;
}

// ------------------------------------------------------------------ learned warm start
int64_t enkf_mlp_param_count(const enkf_mlp_shape* shape) { return enkf::mlp_param_count(shape); }

int64_t enkf_mlp_work_bytes(const enkf_mlp_shape* shape, int32_t batch) {
  return enkf::mlp_work_bytes(shape, batch);
}

enkf_status enkf_mlp_forward(const enkf_mlp_shape* shape, const float* d_params, const float* d_X,
                             const int32_t* d_rows, int32_t batch, float* d_Y, void* d_work,
                             void* cuda_stream) {
  if (enkf::mlp_param_count(shape) < 0 || !d_params || !d_X || !d_Y || !d_work || batch < 1)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_mlp_forward: bad argument");
  cudaError_t e = enkf::mlp_forward(shape, d_params, d_X, d_rows, batch, d_Y, d_work,
                                    static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ENKF_OK : cuda_fail(nullptr, e, "enkf_mlp_forward");
}

enkf_status enkf_mlp_loss_grad(const enkf_mlp_shape* shape, const float* d_params, const float* d_X,
                               const float* d_T, const int32_t* d_rows, int32_t batch,
                               float* d_grad, float* d_loss, void* d_work, void* cuda_stream) {
  if (enkf::mlp_param_count(shape) < 0 || !d_params || !d_X || !d_T || !d_grad || !d_work || batch < 1)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_mlp_loss_grad: bad argument");
  cudaError_t e = enkf::mlp_loss_grad(shape, d_params, d_X, d_T, d_rows, batch, d_grad, d_loss, d_work,
                                      static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ENKF_OK : cuda_fail(nullptr, e, "enkf_mlp_loss_grad");
}

enkf_status enkf_mlp_adam(int64_t count, float* d_params, const float* d_grad, float* d_m, float* d_v,
                          int32_t step, float lr, float beta1, float beta2, float eps, void* cuda_stream) {
  if (count < 1 || !d_params || !d_grad || !d_m || !d_v || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) ||
      !(beta2 >= 0.f && beta2 < 1.f))
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_mlp_adam: bad argument");
  cudaError_t e = enkf::mlp_adam(count, d_params, d_grad, d_m, d_v, step, lr, beta1, beta2, eps,
                                 static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ENKF_OK : cuda_fail(nullptr, e, "enkf_mlp_adam");
}

enkf_status enkf_mlp_train_epoch(const enkf_mlp_shape* shape, float* d_params, float* d_m, float* d_v,
                                 const float* d_X, const float* d_T, const int32_t* d_perm,
                                 int64_t rows, int32_t batch, int32_t step0, float lr,
                                 float* d_losses, float* d_grad, void* d_work, void* cuda_stream) {
  if (enkf::mlp_param_count(shape) < 0 || !d_params || !d_m || !d_v || !d_X || !d_T || !d_perm || !d_grad ||
      !d_work || batch < 1 || rows < batch || step0 < 0)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_mlp_train_epoch: bad argument");
  cudaError_t e = enkf::mlp_train_epoch(shape, d_params, d_m, d_v, d_X, d_T, d_perm, rows, batch, step0, lr,
                                        d_losses, d_work, d_grad, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ENKF_OK : cuda_fail(nullptr, e, "enkf_mlp_train_epoch");
}

enkf_status enkf_mlp_standardize(const enkf_mlp_shape* shape, float* d_params, const float* d_X,
                                 const float* d_T, int64_t rows, void* cuda_stream) {
  if (enkf::mlp_param_count(shape) < 0 || !d_params || !d_X || !d_T || rows < 1)
    return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_mlp_standardize: bad argument");
  cudaError_t e = enkf::mlp_standardize(shape, d_params, d_X, d_T, rows, static_cast<cudaStream_t>(cuda_stream));
  return e == cudaSuccess ? ENKF_OK : cuda_fail(nullptr, e, "enkf_mlp_standardize");
}

enkf_status enkf_warm_features(enkf_handle h, int32_t K, float* d_F, float* d_T) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_warm_features: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_warm_features: batched handle");
  if (h->cfg.precision != ENKF_FP32 || h->cfg.variant != ENKF_CGD)
    return fail(h, ENKF_ERR_UNSUPPORTED, "enkf_warm_features: needs ENKF_CGD in ENKF_FP32");
  if (!h->has_result) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_warm_features: no analysis yet");
  if (K < 1 || !d_F) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_warm_features: K < 1 or NULL d_F");
  cudaError_t e = enkf::warm_features(h, K, d_F, d_T);
  return e == cudaSuccess ? ENKF_OK : cuda_fail(h, e, "enkf_warm_features");
}

enkf_status enkf_set_warm_model(enkf_handle h, const enkf_mlp_shape* shape, const float* d_params) {
  if (!h) return fail(nullptr, ENKF_ERR_INVALID_ARG, "enkf_set_warm_model: NULL handle");
  if (h->batch) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_set_warm_model: batched handle");
  if (h->cfg.precision != ENKF_FP32 || h->cfg.variant != ENKF_CGD)
    return fail(h, ENKF_ERR_UNSUPPORTED, "enkf_set_warm_model: needs ENKF_CGD in ENKF_FP32");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "enkf_set_warm_model");
  if (!d_params) {
    enkf::warm_free(h);
    return ENKF_OK;
  }
  std::string err;
  e = enkf::warm_set_model(h, shape, d_params, err);
  if (e == cudaErrorInvalidValue) return fail(h, ENKF_ERR_INVALID_ARG, "enkf_set_warm_model: " + err);
  if (e != cudaSuccess) return cuda_fail(h, e, ("enkf_set_warm_model: " + err).c_str());
  return ENKF_OK;
}

enkf_status enkf_destroy(enkf_handle h) {
  if (!h) return ENKF_OK;
  cudaStreamSynchronize(h->stream);
  enkf::batch_free(h);
  enkf::warm_free(h);
  for (auto& ev : h->ev)
    if (ev) cudaEventDestroy(ev);
  if (h->copy_stream) {
    cudaStreamSynchronize(h->copy_stream);
    cudaStreamDestroy(h->copy_stream);
  }
  for (auto& ev : h->host_ev)
    if (ev) cudaEventDestroy(ev);
  free_workspace(h->ws);
  delete h;
  return ENKF_OK;
}

}  // extern "C"
