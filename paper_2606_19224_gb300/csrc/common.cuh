// Internal declarations shared by the CUDA translation units of libenkf.so.
// Not part of the public ABI (that is include/enkf.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "enkf.h"

namespace enkf {

constexpr int kThreads = 256;                          // every kernel here uses 256-thread CTAs
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;  // 4 s per grid-barrier wait

// Device status bits (folded into enkf_status by enkf_get_stats).
enum : int { DS_NOT_CONVERGED = 1, DS_NONFINITE = 2, DS_BREAKDOWN = 4, DS_TIMEOUT = 8, DS_SMEM = 16 };

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

// ------------------------------------------------------------------ device helpers
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative (co-resident) launch. `count` is a monotonic arrival
// counter zeroed before the launch; `epoch` is the block's local barrier number. Each wait
// is bounded: after timeout_ns (kBarrierTimeoutNs unless set) the waiting block raises `abort_flag` and the
// DS_TIMEOUT status bit, and every block that sees the flag leaves the barrier with false.
// Returns the same value to all threads of the block.
struct GridBarrier {
  unsigned* count;
  int* abort_flag;
  int* status;
  unsigned nblocks;
  unsigned epoch;
  unsigned long long timeout_ns = kBarrierTimeoutNs;

  __device__ bool sync() {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
      int ok = 1;
      epoch += 1;
      if (nblocks > 1) {
        __threadfence();
        atomicAdd(count, 1u);
        const unsigned target = epoch * nblocks;
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(count) < target) {
          if (*(volatile int*)abort_flag) { ok = 0; break; }
          if (global_ns() - t0 > timeout_ns) {
            atomicExch(abort_flag, 1);
            atomicOr(status, DS_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(20);
        }
        __threadfence();
      } else if (*(volatile int*)abort_flag) {
        ok = 0;
      }
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two 32x32->64-bit
// multiplies by 0xD2511F53 / 0xCD9E8D57 with a Weyl key schedule (0x9E3779B9, 0xBB67AE85).
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
}

// Standard normal for element (i, j) of the perturbation matrix: counter
// (i, j >> 1, ctr_lo, ctr_hi), key (seed_lo, seed_hi); 53-bit uniforms
// u1 = ((w0 << 21 | w1 >> 11) + 0.5) 2^-53, u2 = (w2 << 21 | w3 >> 11) 2^-53; Box-Muller
// radius sqrt(-2 ln u1) times cos(2 pi u2) for even j, sin(2 pi u2) for odd j.
__device__ __forceinline__ double perturbation_normal(int64_t i, int j, uint64_t seed,
                                                      uint64_t counter) {
  uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(j >> 1), c2 = (uint32_t)counter,
           c3 = (uint32_t)(counter >> 32);
  philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t x1 = ((uint64_t)c0 << 21) | (c1 >> 11);
  const uint64_t x2 = ((uint64_t)c2 << 21) | (c3 >> 11);
  const double u1 = ((double)x1 + 0.5) * 0x1p-53;
  const double u2 = (double)x2 * 0x1p-53;
  const double rho = sqrt(-2.0 * log(u1));
  double s, c;
  sincos(6.283185307179586 * u2, &s, &c);
  return rho * ((j & 1) ? s : c);
}

// ------------------------------------------------------------------ host-side state
// Device workspace of one handle. Sizes in elements; all pointers are device pointers.
struct Workspace {
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* w = nullptr;
  double* r = nullptr;          // [m]
  float* r32 = nullptr;         // [m]     (FP32 mode)
  double* HA64 = nullptr;       // [m][N]
  float* HA32 = nullptr;        // [m][N]   (FP32 and mixed modes)
  void* HA16 = nullptr;         // [m][N]   BF16 or FP16 (mixed modes)
  void* HAdf = nullptr;         // [m][N]   double-float HA, D and solution (FP32, mixed modes)
  void* Ddf = nullptr;
  void* Zdf = nullptr;
  double* D = nullptr;          // [m][N]
  double* Z = nullptr;          // [m][N]   FP64 solution (FP64 mode: the CG iterate itself)
  void* B = nullptr;            // [m][N]   inner right-hand side (FP32 mode)
  void* X = nullptr;            // [m][N]   inner iterate (FP32 mode)
  void* Res = nullptr;          // [m][N]
  void* P = nullptr;            // [m][N]
  void* Sv = nullptr;           // [m][N]   S p, carried by the CG recurrences
  double* Tpart = nullptr;      // [G][N*N+2N]
  double* Tred = nullptr;       // [N*N+2N]
  double* rrpart = nullptr;     // [2][G][NT]
  double* Wacc = nullptr;       // [N][N]
  double* W = nullptr;          // [N][N]
  int32_t* col_iters = nullptr; // [N]
  double* col_relres = nullptr; // [N]
  double* col_true = nullptr;   // [N]
  double* col_warm = nullptr;   // [N] true relative residual of a learned start (FP32 mode)
  int32_t* status = nullptr;    // [4]: status bits, refinements, grid, spare
  unsigned* bar = nullptr;      // [4]: barrier counter, abort flag, spare
  void* stage_Xf = nullptr;     // host-API staging [n][N]
  double* stage_y = nullptr;    // [m]
  unsigned long long* prof = nullptr;  // [8] in-kernel phase timers of the solve (ns)
  float* Tk = nullptr;          // [2][N][N] T of the tensor-core step, carried between steps
  double* Tacc = nullptr;       // [3][N N + 4 N] step sums of the tensor-core solve (atomic adds)
  unsigned* hamax = nullptr;    // tensor-core modes: largest |HA| of the analysis (float bits)
  // tridiagonal R (kernels_whiten.cu): the caller's H, the whitening scan's coefficients and
  // buffers; rowptr / col / w / r above then hold H' = I and r' = 1 of the whitened problem
  int32_t* Hrowptr = nullptr;   // [m+1]
  int32_t* Hcol = nullptr;      // [nnz]
  double* Hw = nullptr;         // [nnz]
  double* wa = nullptr;         // [m]   1 / L_ii
  double* wb = nullptr;         // [m]   -L_{i,i-1} / L_ii
  double* wcp = nullptr;        // [m]   product of wb over the scan block up to row i
  double* wmu = nullptr;        // [blocks] product of wb over each scan block
  double* wU = nullptr;         // [m][N+1] anomalies and y - zbar, whitened in place
  double* wV = nullptr;         // [m][N]  explicit perturbations, whitened in place
  double* wcarry = nullptr;     // [blocks][N+1]
  double* wcarryV = nullptr;    // [blocks][N]
  void* Xw = nullptr;           // [m][N]  whitened observed ensemble (FP64 or FP32)
  double* yw = nullptr;         // [m]     whitened y - zbar
};

struct BatchState;   // kernels_batch.cu: plan, arena and graph of a batched handle
struct WarmState;    // kernels_mlp.cu: learned warm-start model and buffers

struct SolveLaunch {
  int G = 0;          // persistent grid size
  int NT = 0;         // padded column tile: 32, 64 or 128
  size_t smem = 0;    // dynamic shared memory per CTA
};

}  // namespace enkf

struct enkf_handle_s {
  enkf_config cfg;
  cudaStream_t stream = nullptr;
  int64_t nnz = 0;
  int device = 0;
  int sms = 0;
  enkf::Workspace ws;
  enkf::SolveLaunch launch;
  std::string last_error;
  bool has_result = false;
  bool timing = false;
  bool timed = false;
  bool prof_enabled = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // enkf_analyze_host with a pinned X_f: the upload of X_f runs on its own stream (created on
  // first use) while the innovations read the observed rows from host memory
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t host_ev[2] = {nullptr, nullptr};
  enkf::BatchState* batch = nullptr;   // non-NULL for a handle made by enkf_batch_create
  enkf::WarmState* warm = nullptr;     // learned warm start (enkf_set_warm_model / enkf_warm_features)
  bool tri = false;                    // tridiagonal R: analyses run on the whitened problem
  float r_pow2 = 1.f;                  // power of two nearest the geometric mean of R's diagonal
                                       // (1 for the whitened problem)
};

namespace enkf {
// Launchers (kernels_fp.cu). Each enqueues on h->stream and returns a cudaError_t.
cudaError_t launch_innovations(enkf_handle_s* h, const void* Xf, const double* y,
                               const double* E, int emode, uint64_t seed, uint64_t counter);
cudaError_t plan_solve(enkf_handle_s* h);
cudaError_t launch_solve(enkf_handle_s* h);
cudaError_t launch_convert_r(enkf_handle_s* h);
// kernels_tc.cu: mixed-precision (BF16 / FP16 tensor-core) persistent solve
cudaError_t plan_solve_mixed(enkf_handle_s* h);
cudaError_t launch_solve_mixed(enkf_handle_s* h);
size_t mixed_image_bytes(const enkf_handle_s* h);   // tile images of HA (zeroed at create)
cudaError_t launch_update(enkf_handle_s* h, const void* Xf, void* Xa);
// kernels_update_tc.cu: X_a = X_f + A W on the tensor cores (FP32 ensembles)
cudaError_t launch_update_tc(enkf_handle_s* h, const void* Xf, void* Xa);
cudaError_t launch_update_product(enkf_handle_s* h, const void* Xf, void* Xa);
// kernels_reduced.cu: Gram pass + N x N CG of CGD-EnKF-Reduced; V lands in ws.W,
// G in ws.Tred, M in ws.Wacc; the CTA partials use ws.Tpart ([reduced_grid][2 N N]).
int reduced_grid(const enkf_handle_s* h);
cudaError_t launch_reduced(enkf_handle_s* h, const void* Xf, const double* y, const double* E,
                           int emode, uint64_t seed, uint64_t counter);
// kernels_batch.cu: batched analyses (planner, arena, persistent kernel, graph, tuner)
struct BatchPlanOut {
  int grid = 0, teams = 0;
  double alpha = 0.0;
  int graphed = 0;
  int row_floors[4] = {0, 0, 0, 0};   // per N class (<= 16, 32, 64, 128): rows per CTA at least
};
bool batch_plan_host(int count, const enkf_config* cfgs, int max_grid, double alpha, const int* row_floors,
                     int* cta_team, int* cta_rank, int* team_size, int* team_first, int* order,
                     BatchPlanOut* out);
cudaError_t batch_build(enkf_handle_s* h, int count, const enkf_config* cfgs,
                        const int32_t* const* rowptr, const int32_t* const* col,
                        const double* const* w, const double* const* r, std::string& err);
cudaError_t batch_analyze(enkf_handle_s* h, const void* const* Xf, const double* const* y,
                          const uint64_t* seeds, const uint64_t* counters, void* const* Xa);
cudaError_t batch_tune(enkf_handle_s* h, const void* const* Xf, const double* const* y,
                       const uint64_t* seeds, const uint64_t* counters, void* const* Xa,
                       double* best_alpha, double* best_ms);
cudaError_t batch_stats(enkf_handle_s* h, int32_t* status, int32_t* iters_max, double* relres_max,
                        int32_t* refinements);
BatchPlanOut batch_info(const enkf_handle_s* h);
// selftest.cu: a bounded wait that nothing releases (failure-detection check)
cudaError_t selftest_wait_timeout(int which, double timeout_ms, cudaStream_t s, int* status_bits);
cudaError_t batch_set_phase_timing(enkf_handle_s* h, bool on);
bool batch_phase_timing(const enkf_handle_s* h);
cudaError_t batch_times(enkf_handle_s* h, double* start_us, double* end_us, double* phase_us, int32_t* team);
int batch_count(const enkf_handle_s* h);
size_t batch_state_bytes(const enkf_handle_s* h, int i);   // bytes of X_f of problem i
void batch_free(enkf_handle_s* h);
// kernels_mlp.cu: the MLP of the learned warm start and its use in an analysis
cudaError_t warm_features(enkf_handle_s* h, int K, float* F, float* T);
cudaError_t warm_set_model(enkf_handle_s* h, const enkf_mlp_shape* shape, const float* params, std::string& err);
bool warm_ready(const enkf_handle_s* h);
cudaError_t warm_prepare(enkf_handle_s* h);
void warm_free(enkf_handle_s* h);
int64_t mlp_param_count(const enkf_mlp_shape* s);
int64_t mlp_work_bytes(const enkf_mlp_shape* s, int B);
cudaError_t mlp_forward(const enkf_mlp_shape* s, const float* P, const float* X, const int32_t* rows, int B,
                        float* Y, void* work, cudaStream_t st);
cudaError_t mlp_loss_grad(const enkf_mlp_shape* s, const float* P, const float* X, const float* T,
                          const int32_t* rows, int B, float* grad, float* loss, void* work, cudaStream_t st);
cudaError_t mlp_adam(int64_t count, float* P, const float* g, float* m, float* v, int step, float lr, float b1,
                     float b2, float eps, cudaStream_t st);
cudaError_t mlp_train_epoch(const enkf_mlp_shape* s, float* P, float* m, float* v, const float* X, const float* T,
                            const int32_t* perm, int64_t rows, int B, int step0, float lr, float* losses,
                            void* work, float* grad, cudaStream_t st);
cudaError_t mlp_standardize(const enkf_mlp_shape* s, float* P, const float* X, const float* T, int64_t rows,
                            cudaStream_t st);
cudaError_t launch_draw_perturbations(uint64_t seed, uint64_t counter, const double* r,
                                      int64_t m, int N, double* E, cudaStream_t s);
// kernels_whiten.cu: tridiagonal R through the whitened problem
bool whiten_coefficients(int64_t m, const double* r, const double* r_off, std::vector<double>& a,
                         std::vector<double>& b, std::vector<double>& cp, std::vector<double>& mu);
int64_t whiten_blocks(int64_t m);
cudaError_t launch_whiten(enkf_handle_s* h, const void* Xf, const double* y, const double* E);
}  // namespace enkf
