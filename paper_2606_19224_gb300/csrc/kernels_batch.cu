// Batched analyses: many independent CGD-EnKF problems of uneven (n, m, N) in one persistent
// cooperative launch, replayed from a CUDA graph. Each problem is the analysis of Fig. 2 /
// Algorithm 1 (innovations, CG solve of S Z = D with the matrix-free product of the
// matvec decomposition, X_a = X_f + A HA^T Z / (N - 1)), in the FP32-with-refresh mode.
//
// Planning (host): a problem is costed at m N^2 (N + 8) + 2 n N^2 (about N preconditioned
// steps of 4 m N^2 flops each, plus the update). The planner minimises the estimated
// makespan: problems costlier than the target get a team of CTAs of their own, the rest wait
// in a queue, longest first (make_plan). Every team works through its problem; for each it
// runs the innovations over its rows, the persistent CG solve with a bounded barrier over the
// team's CTAs only, and the ensemble update, and the team's first CTA stamps the problem's
// start and end. A CTA that is free (outside every team, or its team's problem done) takes
// the next problem of the queue through an atomic counter and solves it alone. The tuner
// times a few values of the team-scaling exponent alpha on the caller's inputs, then
// re-plans from the measured per-problem durations, and keeps the fastest plan; the choice
// can be cached in the text file named by the ENKF_TUNE_CACHE variable.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "innov_device.cuh"
#include "solve_body.cuh"

namespace enkf {

struct BatchProblem {
  SolveParams sp;
  int64_t n;
  int NT;
  const int32_t* rowptr;
  const int32_t* col;
  const double* w;
};
struct BatchIO {
  const float* Xf;
  const double* y;
  float* Xa;
  uint64_t seed, counter;
};

// The per-problem phases as separate (not inlined) device functions, so that each gets the
// register allocation of its own loop nest instead of the union of all of them.
template <int NT>
__device__ __noinline__ void batch_solve(const SolveParams& sp, int G, int rank, GridBarrier& bar,
                                         unsigned char* smem) {
  solve_body<float, NT, true>(sp, G, rank, bar, smem);
}
template <int NT>
__device__ __noinline__ void batch_update(const BatchIO& io, const double* W, int64_t n, int N,
                                          int rank, int G, unsigned char* smem) {
  update_rows<float, NT, 0>(io.Xf, io.Xa, W, n, N, rank, G, smem);
}

// NTMAX bounds the column tile of every problem in the batch. One CTA per SM (the
// double-buffered fused pass takes most of the shared memory). The solve is the
// Jacobi-preconditioned (M = R) form. A CTA first works through its team's list of problems
// (order[team_first[team] .. team_first[team + 1])), then takes problems one at a time from
// the shared queue order[queue_first .. count) (longest first) and solves each alone.
template <int NTMAX>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(
    const BatchProblem* __restrict__ probs, const BatchIO* __restrict__ io,
    const int* __restrict__ cta_team, const int* __restrict__ cta_rank,
    const int* __restrict__ team_size, const int* __restrict__ team_first,
    const int* __restrict__ order, int queue_first, int count, unsigned* __restrict__ queue_head,
    double* __restrict__ team_buf, int max_grid, int ne_max, int perturb,
    unsigned long long* __restrict__ times) {
  constexpr int NT2 = NTMAX >= 64 ? 64 : 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SolveParams s_sp;
  __shared__ BatchIO s_io;
  __shared__ int64_t s_n;
  __shared__ int s_nt;
  __shared__ int s_q;
  const int warp = threadIdx.x >> 5;
  // problem pi on a team of G CTAs in which this CTA has `rank` (the team's CTAs are
  // contiguous, so its reduction slices start at CTA blockIdx.x - rank); false if a barrier
  // of the problem gave up
  auto run = [&](int pi, int G, int rank) -> bool {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_sp = probs[pi].sp;
      const int64_t c0 = (int64_t)blockIdx.x - rank;
      s_sp.Tpart = team_buf + c0 * ne_max;                                      // [G][NE]
      s_sp.Tred = team_buf + (int64_t)max_grid * ne_max + c0 * ne_max;          // [NE]
      s_sp.rrpart = team_buf + (int64_t)2 * max_grid * ne_max + c0 * 256;       // [2][G][NT]
      s_io = io[pi];
      s_n = probs[pi].n;
      s_nt = probs[pi].NT;
      if (rank == 0) times[2 * pi] = global_ns();
    }
    __syncthreads();
    const SolveParams& sp = s_sp;
    const int NT = s_nt;
    GridBarrier bar{sp.bar, reinterpret_cast<int*>(sp.bar + 1), sp.status, (unsigned)G, 0u};
    // innovations over this CTA's block of observation rows (the solve uses the same blocks)
    const int64_t rows_per = (sp.m + G - 1) / G;
    const int64_t r0 = imin64(sp.m, (int64_t)rank * rows_per), r1 = imin64(sp.m, r0 + rows_per);
    innov_rows<float>(s_io.Xf, probs[pi].rowptr, probs[pi].col, probs[pi].w, s_io.y, sp.r, nullptr,
                      perturb ? 2 : 0, s_io.seed, s_io.counter, sp.m, sp.N, nullptr,
                      static_cast<float*>(const_cast<void*>(sp.HA)), const_cast<double*>(sp.D),
                      static_cast<float*>(sp.B), nullptr, nullptr, 0, const_cast<df32*>(sp.HAdf),
                      const_cast<df32*>(sp.Ddf), r0, r1, warp, kThreads / 32);
    bool ok = bar.sync();
    if (ok) {
      if (NT == 32) batch_solve<32>(sp, G, rank, bar, smem);
      else if (NT == 64) batch_solve<NT2>(sp, G, rank, bar, smem);
      else batch_solve<NTMAX>(sp, G, rank, bar, smem);
      ok = bar.sync();   // W of this problem complete and visible to the team
    }
    if (!ok) return false;
    if (NT == 32) batch_update<32>(s_io, sp.W, s_n, sp.N, rank, G, smem);
    else if (NT == 64) batch_update<NT2>(s_io, sp.W, s_n, sp.N, rank, G, smem);
    else batch_update<NTMAX>(s_io, sp.W, s_n, sp.N, rank, G, smem);
    __syncthreads();
    if (rank == 0 && threadIdx.x == 0) times[2 * pi + 1] = global_ns();
    return true;
  };
  const int team = cta_team[blockIdx.x], rank = cta_rank[blockIdx.x], G = team_size[team];
  const int k_end = team_first[team + 1];
  for (int k = team_first[team]; k < k_end; ++k) {
    if (!run(order[k], G, rank)) {
      // a barrier gave up: the team is no longer in step, so it leaves its list here and
      // flags the problems it has not finished; its CTAs still serve the queue alone
      if (rank == 0 && threadIdx.x == 0)
        for (int q = k; q < k_end; ++q) atomicOr(probs[order[q]].sp.status, DS_TIMEOUT);
      break;
    }
  }
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_q = queue_first + (int)atomicAdd(queue_head, 1u);
    __syncthreads();
    const int q = s_q;
    if (q >= count) break;
    run(order[q], 1, 0);   // one CTA: its barriers never wait
  }
}

// ------------------------------------------------------------------ host side
// Row-block floor per ensemble-size class (N <= 16, <= 32, <= 64, <= 128): a team of k CTAs
// for a problem of m rows needs m / k >= floor rows per CTA, which caps the team at
// ceil(m / floor) CTAs. The tuner searches it per class (64 .. 512 rows).
constexpr int kNClasses = 4;
using RowFloors = std::array<int, kNClasses>;
constexpr RowFloors kDefaultFloors{64, 64, 64, 64};
static int n_class(int N) { return N <= 16 ? 0 : (N <= 32 ? 1 : (N <= 64 ? 2 : 3)); }

struct BatchPlan {
  double alpha = 1.0;
  RowFloors floors = kDefaultFloors;
  std::vector<double> cost;   // per-problem one-CTA cost the plan was made from
  bool measured = false;      // cost holds measured times (ns) instead of the model's
  int grid = 0;
  std::vector<int> cta_team, cta_rank, team_size, team_first, order, team_cta0;
  int queue_first = 0;        // order[queue_first ..] is the shared queue
};

struct BatchState {
  int count = 0;
  int perturb = 1;
  int ntmax = 32;
  int ne_max = 0;
  size_t smem = 0;
  int max_grid = 0;
  std::vector<enkf_config> cfg;
  void* arena = nullptr;
  std::vector<BatchProblem> probs;     // host copy (device pointers into the arena)
  BatchProblem* d_probs = nullptr;
  BatchIO* d_io = nullptr;
  BatchIO* h_io = nullptr;             // pinned staging of the per-call table
  std::vector<BatchIO> last_io;        // table currently on the device
  cudaEvent_t io_copied = nullptr;     // the last table upload has finished reading h_io
  int* d_plan = nullptr;               // cta_team | cta_rank | team_size | team_first | order
                                       // (grid, grid, teams, teams + 1, count entries)
  int* d_status = nullptr;             // [count][4]: status bits, refinements
  unsigned* d_bar = nullptr;           // [count][4]: barrier counter, abort flag; then the queue head
  double* d_team = nullptr;            // Tpart [max_grid][NE], Tred [max_grid][NE], rrpart [max_grid][256]
  unsigned long long* d_time = nullptr;   // [count][2]: start, end (global ns, by each team's rank 0)
  unsigned long long* d_phase = nullptr;  // [count][PH_COUNT] solve phase timers, or nullptr when off
  BatchPlan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graph_ok = true;                // capture works here; else launches go direct
};

static int nt_of(int N) { return N <= 32 ? 32 : (N <= 64 ? 64 : 128); }

static double problem_cost(const enkf_config& c) {
  const double m = (double)c.m, N = c.N, n = (double)c.n;
  return m * N * N * (N + 8.0) + 2.0 * n * N * N;
}

// Makespan planning. A team of k CTAs is assumed to finish a problem of cost c in c / k^alpha
// (alpha <= 1 charges large teams for their barriers and reductions). For a target time T,
// every problem with c > T gets the smallest team that meets T (at most ceil(m / floor) CTAs,
// floor the row-block floor of its N class); the others form the shared queue, longest first. The queue is
// simulated as the kernel serves it: the next problem goes to the CTA that is free first
// (the CTAs outside teams at time 0, each team's CTAs when its problem is done), and every
// problem must end by T. The plan is the one for the smallest feasible T (bisection); CTAs
// the queue cannot use then join the slowest teams.
struct PlanTeam {
  int size;
  double load;   // estimated time
  std::vector<int> probs;
};
struct PlanTry {
  std::vector<PlanTeam> teams;   // multi-CTA teams, one problem each
  std::vector<int> queue;        // the other problems, costs descending
  int free_ctas = 0;             // CTAs outside teams
};

static bool try_plan(const std::vector<double>& cost, const std::vector<int>& cap, const std::vector<int>& idx,
                     int G, double alpha, double T, PlanTry* out) {
  PlanTry o;
  int used = 0;
  for (int pi : idx) {   // costs descending
    if (cost[pi] > T) {
      int k = (int)std::ceil(std::pow(cost[pi] / T, 1.0 / alpha) - 1e-9);
      k = std::max(k, 2);
      if (k > cap[pi]) return false;
      used += k;
      if (used > G) return false;
      o.teams.push_back({k, cost[pi] / std::pow((double)k, alpha), {pi}});
    } else {
      o.queue.push_back(pi);
    }
  }
  o.free_ctas = G - used;
  if (!o.queue.empty()) {
    std::priority_queue<double, std::vector<double>, std::greater<double>> avail;
    for (int q = 0; q < o.free_ctas; ++q) avail.push(0.0);
    for (const PlanTeam& t : o.teams)
      for (int r = 0; r < t.size; ++r) avail.push(t.load);
    for (int pi : o.queue) {
      const double f = avail.top() + cost[pi];
      if (f > T * (1.0 + 1e-12)) return false;
      avail.pop();
      avail.push(f);
    }
  }
  if (out) *out = std::move(o);
  return true;
}

// cost[i]: the estimated time of problem i on one CTA (problem_cost, or a measurement).
static BatchPlan make_plan(const std::vector<enkf_config>& cfg, const std::vector<double>& cost, int G,
                           double alpha, const RowFloors& floors = kDefaultFloors) {
  BatchPlan P;
  P.alpha = alpha;
  P.floors = floors;
  P.cost = cost;
  const int count = (int)cfg.size();
  std::vector<int> cap(count);
  for (int i = 0; i < count; ++i) {
    const int64_t fl = floors[n_class(cfg[i].N)];
    cap[i] = (int)std::max<int64_t>(1, std::min<int64_t>(G, (cfg[i].m + fl - 1) / fl));
  }
  std::vector<int> idx(count);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  // bisection on the makespan T between a lower bound and a target that always fits
  const double total = std::accumulate(cost.begin(), cost.end(), 0.0);
  double lo = total / G;
  for (int i = 0; i < count; ++i) lo = std::max(lo, cost[i] / std::pow((double)cap[i], alpha));
  double hi = total + 1.0;   // every problem in the queue: fits on one CTA
  PlanTry best;
  try_plan(cost, cap, idx, G, alpha, hi, &best);
  for (int it = 0; it < 60 && hi > lo * (1.0 + 1e-6); ++it) {
    const double mid = 0.5 * (lo + hi);
    PlanTry trial;
    if (try_plan(cost, cap, idx, G, alpha, mid, &trial)) {
      hi = mid;
      best = std::move(trial);
    } else {
      lo = mid;
    }
  }
  // CTAs beyond what the queue can keep busy join the slowest teams
  int spare = best.free_ctas - (int)best.queue.size();
  for (; spare > 0; --spare) {
    int w = -1;
    for (int q = 0; q < (int)best.teams.size(); ++q) {
      const PlanTeam& t = best.teams[q];
      if (t.size >= cap[t.probs[0]]) continue;
      if (w < 0 || t.load > best.teams[w].load) w = q;
    }
    if (w < 0) break;
    PlanTeam& t = best.teams[w];
    t.size += 1;
    t.load = cost[t.probs[0]] / std::pow((double)t.size, alpha);
    best.free_ctas -= 1;
  }
  // multi-CTA teams with their problem, then the free CTAs as teams of one with empty lists;
  // order ends with the queue
  int cta = 0;
  P.team_first.push_back(0);
  auto add_team = [&](int size, const std::vector<int>& probs) {
    const int tid = (int)P.team_size.size();
    P.team_size.push_back(size);
    P.team_cta0.push_back(cta);
    for (int r = 0; r < size; ++r) {
      P.cta_team.push_back(tid);
      P.cta_rank.push_back(r);
    }
    cta += size;
    for (int pi : probs) P.order.push_back(pi);
    P.team_first.push_back((int)P.order.size());
  };
  for (const PlanTeam& t : best.teams) add_team(t.size, t.probs);
  const int nfree = std::min(best.free_ctas, std::max(0, (int)best.queue.size()));
  for (int q = 0; q < nfree; ++q) add_team(1, {});
  if (cta == 0) add_team(1, {});   // a grid of at least one CTA
  P.queue_first = (int)P.order.size();
  for (int pi : best.queue) P.order.push_back(pi);
  P.grid = cta;
  return P;
}

static std::vector<double> model_costs(const std::vector<enkf_config>& cfg) {
  std::vector<double> cost(cfg.size());
  for (size_t i = 0; i < cfg.size(); ++i) cost[i] = problem_cost(cfg[i]);
  return cost;
}

bool batch_plan_host(int count, const enkf_config* cfgs, int max_grid, double alpha, const int* row_floors,
                     int* cta_team, int* cta_rank, int* team_size, int* team_first, int* order,
                     BatchPlanOut* out) {
  if (count < 1 || !cfgs || max_grid < 1) return false;
  const std::vector<enkf_config> cfg(cfgs, cfgs + count);
  RowFloors fl = kDefaultFloors;
  if (row_floors)
    for (int c = 0; c < kNClasses; ++c) fl[c] = row_floors[c];
  const BatchPlan P = make_plan(cfg, model_costs(cfg), max_grid, alpha, fl);
  auto put = [](const std::vector<int>& v, int* dst) { if (dst) std::copy(v.begin(), v.end(), dst); };
  put(P.cta_team, cta_team);
  put(P.cta_rank, cta_rank);
  put(P.team_size, team_size);
  put(P.team_first, team_first);
  put(P.order, order);
  if (out) *out = BatchPlanOut{P.grid, (int)P.team_size.size(), P.alpha, 0, {P.floors[0], P.floors[1], P.floors[2], P.floors[3]}};
  return true;
}

// Dynamic shared memory of a batch whose tiles go up to NTMAX: the largest need of any
// column tile it may run (the NT = 32 and 64 solves use the double-buffered fused pass and
// need more than the NT = 128 one).
template <int NT>
static size_t tile_smem() {
  return std::max<size_t>(solve_smem_bytes<float, NT>(), update_smem_bytes<float, NT>());
}
template <int NTMAX>
static size_t batch_smem_nt() {
  size_t s = tile_smem<32>();
  if (NTMAX >= 64) s = std::max(s, tile_smem<64>());
  if (NTMAX >= 128) s = std::max(s, tile_smem<128>());
  return s;
}

static void* batch_fn(int ntmax) {
  if (ntmax == 32) return (void*)batch_kernel<32>;
  if (ntmax == 64) return (void*)batch_kernel<64>;
  return (void*)batch_kernel<128>;
}

static void drop_graph(BatchState& B) {
  if (B.gexec) { cudaGraphExecDestroy(B.gexec); B.gexec = nullptr; }
  if (B.graph) { cudaGraphDestroy(B.graph); B.graph = nullptr; }
}

// Install a plan: plan arrays and the problem table on the device.
static cudaError_t apply_plan(BatchState& B, const BatchPlan& P, cudaStream_t s) {
  B.plan = P;
  std::vector<int> flat;
  for (const auto* v : {&P.cta_team, &P.cta_rank, &P.team_size, &P.team_first, &P.order})
    flat.insert(flat.end(), v->begin(), v->end());
  drop_graph(B);
  cudaError_t e = cudaStreamSynchronize(s);   // no replay of the old plan is still reading
  if (e == cudaSuccess)
    e = cudaMemcpy(B.d_plan, flat.data(), flat.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(B.d_probs, B.probs.data(), B.probs.size() * sizeof(BatchProblem), cudaMemcpyHostToDevice);
  return e;
}

static cudaError_t enqueue_batch(BatchState& B, cudaStream_t s) {
  const BatchPlan& P = B.plan;
  const int nC = (int)P.cta_team.size(), nT = (int)P.team_size.size();
  int* cta_team = B.d_plan;
  int* cta_rank = cta_team + nC;
  int* team_size = cta_rank + nC;
  int* team_first = team_size + nT;
  int* order = team_first + nT + 1;
  cudaError_t e = cudaMemsetAsync(B.d_bar, 0, sizeof(unsigned) * (4 * (size_t)B.count + 4), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B.d_status, 0, sizeof(int) * 4 * B.count, s);
  if (e != cudaSuccess) return e;
  const BatchProblem* probs = B.d_probs;
  const BatchIO* io = B.d_io;
  int perturb = B.perturb;
  unsigned long long* times = B.d_time;
  int queue_first = P.queue_first, count = B.count, max_grid = B.max_grid, ne_max = B.ne_max;
  unsigned* queue_head = B.d_bar + 4 * (size_t)B.count;
  double* team_buf = B.d_team;
  void* args[] = {&probs, &io, &cta_team, &cta_rank, &team_size, &team_first, &order, &queue_first, &count,
                  &queue_head, &team_buf, &max_grid, &ne_max, &perturb, &times};
  return cudaLaunchCooperativeKernel(batch_fn(B.ntmax), dim3(P.grid), dim3(kThreads), args,
                                     B.smem, s);
}

// One batched analysis: upload the per-call table if it changed, then replay the graph
// (captured on first use after each plan change).
static cudaError_t run_batch(enkf_handle_s* h, const std::vector<BatchIO>& io) {
  BatchState& B = *h->batch;
  cudaError_t e = cudaSuccess;
  const bool same = B.last_io.size() == io.size() &&
                    std::memcmp(B.last_io.data(), io.data(), io.size() * sizeof(BatchIO)) == 0;
  if (!same) {
    e = cudaEventSynchronize(B.io_copied);   // the previous upload no longer reads h_io
    if (e != cudaSuccess) return e;
    std::memcpy(B.h_io, io.data(), io.size() * sizeof(BatchIO));
    e = cudaMemcpyAsync(B.d_io, B.h_io, io.size() * sizeof(BatchIO), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(B.io_copied, h->stream);
    if (e != cudaSuccess) return e;
    B.last_io = io;
  }
  if (!B.graph_ok) return enqueue_batch(B, h->stream);
  if (!B.gexec) {
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t le = enqueue_batch(B, cap);
      e = cudaStreamEndCapture(cap, &B.graph);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B.gexec, B.graph, 0);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      // capture of a cooperative launch refused: the graph is an optimisation, so clear the
      // error and launch the same work directly from now on
      cudaGetLastError();
      drop_graph(B);
      B.graph_ok = false;
      return enqueue_batch(B, h->stream);
    }
  }
  return cudaGraphLaunch(B.gexec, h->stream);
}

static std::string cache_key(const BatchState& B) {
  std::string key = std::to_string(B.count) + ":" + std::to_string(B.max_grid) + ":";
  for (const auto& c : B.cfg)
    key += std::to_string(c.n) + "/" + std::to_string(c.m) + "/" + std::to_string(c.N) + ",";
  return key;
}

// ------------------------------------------------------------------ entry-point helpers
cudaError_t batch_build(enkf_handle_s* h, int count, const enkf_config* cfgs,
                        const int32_t* const* rowptr, const int32_t* const* col,
                        const double* const* w, const double* const* r, std::string& err) {
  auto* Bp = new BatchState();
  h->batch = Bp;
  BatchState& B = *Bp;
  B.count = count;
  B.perturb = cfgs[0].perturb_obs;
  int nmax = 2;
  for (int i = 0; i < count; ++i) {
    B.cfg.push_back(cfgs[i]);
    nmax = std::max(nmax, (int)cfgs[i].N);
  }
  B.ntmax = nt_of(nmax);
  B.ne_max = nmax * nmax + 4 * nmax;
  B.smem = B.ntmax == 32 ? batch_smem_nt<32>() : B.ntmax == 64 ? batch_smem_nt<64>() : batch_smem_nt<128>();
  void* fn = batch_fn(B.ntmax);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, B.smem);
  if (e != cudaSuccess) { err = "enkf_batch_create: occupancy query"; return e; }
  if (occ < 1) { err = "enkf_batch_create: kernel does not fit on an SM"; return cudaErrorInvalidConfiguration; }
  B.max_grid = occ * h->sms;
  if (h->cfg.grid_blocks > 0) B.max_grid = std::min(B.max_grid, h->cfg.grid_blocks);
  // one arena: per problem HA, HAdf, D, Ddf, Zdf, B, X, Res, P, Sv, r, r32, rowptr, col, w,
  // W, column iterations / residuals
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  std::vector<std::vector<size_t>> parts(count);
  std::vector<size_t> off(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    const auto& c = cfgs[i];
    const size_t mN = (size_t)c.m * c.N, m = (size_t)c.m, N = (size_t)c.N;
    const size_t nnz = (size_t)std::max(1, rowptr[i][c.m]);
    parts[i] = {4 * mN, 8 * mN, 8 * mN, 8 * mN, 8 * mN, 4 * mN, 4 * mN, 4 * mN, 4 * mN, 4 * mN,
                8 * m, 4 * m, 4 * (m + 1), 4 * nnz, 8 * nnz, 8 * N * N, 4 * N, 8 * N, 8 * N};
    size_t sz = 0;
    for (size_t b : parts[i]) sz += al(b);
    off[i + 1] = off[i] + sz;
  }
  const size_t NE = (size_t)B.ne_max;
  e = cudaMalloc(&B.arena, off[count]);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_probs, sizeof(BatchProblem) * count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_io, sizeof(BatchIO) * count);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&B.h_io, sizeof(BatchIO) * count);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B.io_copied, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_plan, sizeof(int) * (4 * (size_t)B.max_grid + 1 + count));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_status, sizeof(int) * 4 * count);
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_bar, sizeof(unsigned) * (4 * (size_t)count + 4));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_time, sizeof(unsigned long long) * 2 * count);
  if (e == cudaSuccess) e = cudaMemset(B.d_time, 0, sizeof(unsigned long long) * 2 * count);
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&B.d_team, sizeof(double) * (2 * (size_t)B.max_grid * NE + (size_t)B.max_grid * 256));
  if (e != cudaSuccess) { err = "enkf_batch_create: device allocation"; return e; }
  unsigned char* base = static_cast<unsigned char*>(B.arena);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const auto& c = cfgs[i];
    unsigned char* q = base + off[i];
    std::vector<void*> ptr;
    for (size_t b : parts[i]) { ptr.push_back(q); q += al(b); }
    BatchProblem bp{};
    SolveParams& sp = bp.sp;
    sp.m = c.m;
    sp.N = c.N;
    sp.mode = 1;
    sp.HA = ptr[0];
    sp.HA64 = nullptr;
    sp.HAdf = static_cast<const df32*>(ptr[1]);
    sp.D = static_cast<const double*>(ptr[2]);
    sp.Ddf = static_cast<const df32*>(ptr[3]);
    sp.Zdf = static_cast<df32*>(ptr[4]);
    sp.B = ptr[5];
    sp.X = ptr[6];
    sp.Res = ptr[7];
    sp.P = ptr[8];
    sp.Sv = ptr[9];
    sp.Z = nullptr;
    sp.r = static_cast<const double*>(ptr[10]);
    sp.rv = ptr[11];
    sp.W = static_cast<double*>(ptr[15]);
    sp.col_iters = static_cast<int*>(ptr[16]);
    sp.col_relres = static_cast<double*>(ptr[17]);
    sp.col_true = static_cast<double*>(ptr[18]);
    sp.tol = c.tol;
    sp.inner_tol = c.inner_tol;
    sp.max_iter = c.max_iter;
    sp.fixed_iters = 0;
    sp.max_refine = c.max_refine;
    sp.true_residual = c.true_residual;
    sp.status = B.d_status + 4 * i;
    sp.bar = B.d_bar + 4 * i;
    sp.prof = nullptr;
    bp.n = c.n;
    bp.NT = nt_of(c.N);
    bp.rowptr = static_cast<const int32_t*>(ptr[12]);
    bp.col = static_cast<const int32_t*>(ptr[13]);
    bp.w = static_cast<const double*>(ptr[14]);
    const int64_t nnz = rowptr[i][c.m];
    e = cudaMemcpy(ptr[12], rowptr[i], 4 * ((size_t)c.m + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(ptr[13], col[i], 4 * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && nnz > 0) e = cudaMemcpy(ptr[14], w[i], 8 * (size_t)nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ptr[10], r[i], 8 * (size_t)c.m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
      std::vector<float> r32(c.m);
      for (int64_t k = 0; k < c.m; ++k) r32[k] = (float)r[i][k];
      e = cudaMemcpy(ptr[11], r32.data(), 4 * (size_t)c.m, cudaMemcpyHostToDevice);
    }
    B.probs.push_back(bp);
  }
  if (e != cudaSuccess) { err = "enkf_batch_create: upload of the observation operators"; return e; }
  // a tuning result for this batch: "key alpha [rows f_0 .. f_3] [cost_0 .. cost_{count-1}]"
  // (row-block floors per N class, measured one-CTA costs); the last one wins
  double alpha = 1.0;
  RowFloors floors = kDefaultFloors;
  std::vector<double> cost = model_costs(B.cfg);
  bool measured = false;
  if (const char* path = std::getenv("ENKF_TUNE_CACHE")) {
    std::ifstream f(path);
    const std::string key = cache_key(B);
    std::string line;
    while (std::getline(f, line)) {
      std::istringstream ls(line);
      std::string k;
      double a = 0.0;
      if (!(ls >> k >> a) || k != key || !(a > 0.0 && a <= 1.0)) continue;
      RowFloors fl = kDefaultFloors;
      std::vector<double> c;
      std::string tok;
      bool ok_f = true;
      while (ls >> tok) {
        if (tok == "rows" && c.empty()) {
          for (int q = 0; q < kNClasses && ok_f; ++q) ok_f = static_cast<bool>(ls >> fl[q]) && fl[q] >= 1;
        } else {
          char* end = nullptr;
          const double v = std::strtod(tok.c_str(), &end);
          if (end == tok.c_str() || *end != '\0') { ok_f = false; break; }
          c.push_back(v);
        }
      }
      const bool ok_c = (int)c.size() == count &&
                        std::all_of(c.begin(), c.end(), [](double x) { return x > 0.0 && std::isfinite(x); });
      if (!ok_f || (!c.empty() && !ok_c)) continue;
      alpha = a;
      floors = fl;
      measured = !c.empty();
      cost = measured ? c : model_costs(B.cfg);
    }
  }
  BatchPlan P = make_plan(B.cfg, cost, B.max_grid, alpha, floors);
  P.measured = measured;
  e = apply_plan(B, P, h->stream);
  if (e != cudaSuccess) err = "enkf_batch_create: plan upload";
  return e;
}

static std::vector<BatchIO> make_io(const BatchState& B, const void* const* Xf, const double* const* y,
                                    const uint64_t* seeds, const uint64_t* counters, void* const* Xa) {
  std::vector<BatchIO> io(B.count);
  for (int i = 0; i < B.count; ++i)
    io[i] = BatchIO{static_cast<const float*>(Xf[i]), y[i], static_cast<float*>(Xa[i]),
                    seeds ? seeds[i] : 0, counters ? counters[i] : 0};
  return io;
}

cudaError_t batch_analyze(enkf_handle_s* h, const void* const* Xf, const double* const* y,
                          const uint64_t* seeds, const uint64_t* counters, void* const* Xa) {
  return run_batch(h, make_io(*h->batch, Xf, y, seeds, counters, Xa));
}

// Per-problem durations (ns) of the last analysis, from the start/end stamps of each team's
// rank 0; team size of every problem under plan P.
static cudaError_t problem_ns(const BatchState& B, cudaStream_t s, std::vector<double>& ns) {
  std::vector<unsigned long long> t(2 * (size_t)B.count);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.data(), B.d_time, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost);
  ns.assign(B.count, 0.0);
  for (int i = 0; i < B.count && e == cudaSuccess; ++i)
    ns[i] = t[2 * i + 1] > t[2 * i] ? (double)(t[2 * i + 1] - t[2 * i]) : 0.0;
  return e;
}

static std::vector<int> problem_team(const BatchPlan& P, int count) {
  std::vector<int> k(count, 1);
  for (size_t t = 0; t < P.team_size.size(); ++t)
    for (int q = P.team_first[t]; q < P.team_first[t + 1]; ++q) k[P.order[q]] = P.team_size[t];
  return k;
}

// The tuner. Stage 1 times the model-cost plans for alpha in {1, 0.9, 0.8}. Stage 2 replaces
// the model by measurement, starting from the alpha = 1 plan and from the stage-1 winner if
// that is another: each problem's one-CTA cost is estimated from its duration in the start
// plan (the mean over its three timed analyses, times k^alpha for a team of k), the batch is
// re-planned from those costs and timed, and the estimate is averaged with the new plan's
// durations for the next of four rounds. Stage 3 searches the row-block floor of each N
// class (below). The fastest plan of all is kept.
cudaError_t batch_tune(enkf_handle_s* h, const void* const* Xf, const double* const* y,
                       const uint64_t* seeds, const uint64_t* counters, void* const* Xa,
                       double* best_alpha, double* best_ms) {
  BatchState& B = *h->batch;
  const std::vector<BatchIO> io = make_io(B, Xf, y, seeds, counters, Xa);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // install P, one warm-up analysis (captures the graph), three timed; mean ms and the mean
  // per-problem durations over the three
  auto time_plan = [&](const BatchPlan& P, double& ms_mean, std::vector<double>& ns) {
    cudaError_t r = apply_plan(B, P, h->stream);
    if (r == cudaSuccess) r = run_batch(h, io);
    float tot = 0.f;
    ns.assign(B.count, 0.0);
    std::vector<double> one;
    for (int rep = 0; rep < 3 && r == cudaSuccess; ++rep) {
      float ms = 0.f;
      r = cudaEventRecord(e0, h->stream);
      if (r == cudaSuccess) r = run_batch(h, io);
      if (r == cudaSuccess) r = cudaEventRecord(e1, h->stream);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
      if (r == cudaSuccess) r = problem_ns(B, h->stream, one);
      for (int i = 0; i < B.count && r == cudaSuccess; ++i) ns[i] += one[i] / 3.0;
      tot += ms;
    }
    ms_mean = tot / 3.0;
    return r;
  };
  BatchPlan best_plan = B.plan;
  double best = 1e300;
  const std::vector<double> model = model_costs(B.cfg);
  struct Start { BatchPlan plan; std::vector<double> ns; double ms; };
  std::vector<Start> stage1;
  for (double a : {1.0, 0.9, 0.8}) {
    if (e != cudaSuccess) break;
    Start st{make_plan(B.cfg, model, B.max_grid, a), {}, 0.0};
    e = time_plan(st.plan, st.ms, st.ns);
    if (e != cudaSuccess) break;
    if (st.ms < best) { best = st.ms; best_plan = st.plan; }
    stage1.push_back(std::move(st));
  }
  // measured-cost rounds from the alpha = 1 plan and, if another alpha won stage 1, from that
  // plan too (which model plan wins is itself noisy, and each start converges differently)
  std::vector<size_t> starts;
  if (e == cudaSuccess) {
    size_t win = 0;
    for (size_t q = 1; q < stage1.size(); ++q)
      if (stage1[q].ms < stage1[win].ms) win = q;
    starts.push_back(0);
    if (win != 0) starts.push_back(win);
  }
  for (size_t sidx : starts) {
    if (e != cudaSuccess) break;
    const double a = stage1[sidx].plan.alpha;
    auto one_cta = [&](const BatchPlan& P, const std::vector<double>& ns) {
      const std::vector<int> k = problem_team(P, B.count);
      std::vector<double> c(B.count);
      for (int i = 0; i < B.count; ++i) c[i] = std::max(1.0, ns[i]) * std::pow((double)k[i], a);
      return c;
    };
    std::vector<double> est = one_cta(stage1[sidx].plan, stage1[sidx].ns);
    for (int round = 0; round < 4 && e == cudaSuccess; ++round) {
      BatchPlan P = make_plan(B.cfg, est, B.max_grid, a);
      P.measured = true;
      double ms = 0.0;
      std::vector<double> ns;
      e = time_plan(P, ms, ns);
      if (e != cudaSuccess) break;
      if (ms < best) { best = ms; best_plan = P; }
      const std::vector<double> now = one_cta(P, ns);
      for (int i = 0; i < B.count; ++i) est[i] = 0.5 * (est[i] + now[i]);
    }
  }
  // Stage 3: the row-block floor of each N class (the smallest row block a team's CTA may
  // get, which caps the team size), by coordinate descent from the best plan with its costs
  // and alpha: classes in order of their share of the cost (those under 5 % left at 64 rows),
  // each floor in {128, 256, 512} planned and, where the plan changes, timed; a floor is kept
  // when the batch is at least 1 % faster.
  if (e == cudaSuccess) {
    std::array<double, kNClasses> share{};
    double total = 0.0;
    for (int i = 0; i < B.count; ++i) {
      share[n_class(B.cfg[i].N)] += best_plan.cost[i];
      total += best_plan.cost[i];
    }
    std::array<int, kNClasses> cls{0, 1, 2, 3};
    std::sort(cls.begin(), cls.end(), [&](int a, int b) { return share[a] > share[b]; });
    for (int c : cls) {
      if (e != cudaSuccess || !(share[c] >= 0.05 * total)) continue;
      for (int fl : {128, 256, 512}) {
        RowFloors f = best_plan.floors;
        f[c] = fl;
        BatchPlan P = make_plan(B.cfg, best_plan.cost, B.max_grid, best_plan.alpha, f);
        P.measured = best_plan.measured;
        if (P.team_size == best_plan.team_size && P.order == best_plan.order) continue;   // same plan
        double ms = 0.0;
        std::vector<double> ns;
        e = time_plan(P, ms, ns);
        if (e != cudaSuccess) break;
        if (ms < 0.99 * best) { best = ms; best_plan = P; }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  e = apply_plan(B, best_plan, h->stream);
  if (best_alpha) *best_alpha = best_plan.alpha;
  if (best_ms) *best_ms = best;
  if (const char* path = std::getenv("ENKF_TUNE_CACHE")) {
    std::ofstream f(path, std::ios::app);
    f << cache_key(B) << " " << best_plan.alpha << " rows";
    for (int q = 0; q < kNClasses; ++q) f << " " << best_plan.floors[q];
    if (best_plan.measured) {
      char buf[32];
      for (double c : best_plan.cost) {
        std::snprintf(buf, sizeof(buf), " %.6g", c);
        f << buf;
      }
    }
    f << "\n";
  }
  return e;
}

cudaError_t batch_stats(enkf_handle_s* h, int32_t* status, int32_t* iters_max, double* relres_max,
                        int32_t* refinements) {
  BatchState& B = *h->batch;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  std::vector<int> st(4 * (size_t)B.count);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), B.d_status, sizeof(int) * 4 * B.count, cudaMemcpyDeviceToHost);
  for (int i = 0; i < B.count && e == cudaSuccess; ++i) {
    const SolveParams& sp = B.probs[i].sp;
    const int N = B.cfg[i].N;
    std::vector<int> it(N);
    std::vector<double> rel(N);
    e = cudaMemcpy(it.data(), sp.col_iters, sizeof(int) * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(rel.data(), sp.col_relres, sizeof(double) * N, cudaMemcpyDeviceToHost);
    const int bits = st[4 * (size_t)i];
    int s = ENKF_OK;
    if (bits & DS_SMEM) s = ENKF_ERR_CUDA;
    else if (bits & DS_TIMEOUT) s = ENKF_ERR_TIMEOUT;
    else if (bits & DS_NONFINITE) s = ENKF_ERR_NONFINITE;
    else if (bits & DS_BREAKDOWN) s = ENKF_ERR_BREAKDOWN;
    else if (bits & DS_NOT_CONVERGED) s = ENKF_ERR_NOT_CONVERGED;
    if (status) status[i] = s;
    if (iters_max) iters_max[i] = *std::max_element(it.begin(), it.end());
    if (relres_max) relres_max[i] = *std::max_element(rel.begin(), rel.end());
    if (refinements) refinements[i] = st[4 * (size_t)i + 1];
  }
  return e;
}

cudaError_t batch_set_phase_timing(enkf_handle_s* h, bool on) {
  BatchState& B = *h->batch;
  cudaError_t e = cudaSuccess;
  if (on && !B.d_phase) {
    const size_t bytes = sizeof(unsigned long long) * PH_COUNT * (size_t)B.count;
    e = cudaMalloc((void**)&B.d_phase, bytes);
    if (e == cudaSuccess) e = cudaMemset(B.d_phase, 0, bytes);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < B.count; ++i) B.probs[i].sp.prof = on ? B.d_phase + (size_t)PH_COUNT * i : nullptr;
  const BatchPlan P = B.plan;
  return apply_plan(B, P, h->stream);   // uploads the problem table, recaptures the graph
}

bool batch_phase_timing(const enkf_handle_s* h) { return h->batch->count > 0 && h->batch->probs[0].sp.prof; }

cudaError_t batch_times(enkf_handle_s* h, double* start_us, double* end_us, double* phase_us, int32_t* team) {
  BatchState& B = *h->batch;
  std::vector<unsigned long long> t(2 * (size_t)B.count);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.data(), B.d_time, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && phase_us) {
    std::vector<unsigned long long> ph((size_t)PH_COUNT * B.count);
    e = cudaMemcpy(ph.data(), B.d_phase, sizeof(unsigned long long) * ph.size(), cudaMemcpyDeviceToHost);
    for (size_t q = 0; q < ph.size() && e == cudaSuccess; ++q) phase_us[q] = 1e-3 * (double)ph[q];
  }
  if (e != cudaSuccess) return e;
  unsigned long long t0 = ~0ull;
  for (int i = 0; i < B.count; ++i) t0 = std::min(t0, t[2 * i]);
  for (int i = 0; i < B.count; ++i) {
    if (start_us) start_us[i] = 1e-3 * (double)(t[2 * i] - t0);
    if (end_us) end_us[i] = t[2 * i + 1] >= t[2 * i] ? 1e-3 * (double)(t[2 * i + 1] - t0) : -1.0;
  }
  if (team) {
    const std::vector<int> k = problem_team(B.plan, B.count);
    std::copy(k.begin(), k.end(), team);
  }
  return e;
}

BatchPlanOut batch_info(const enkf_handle_s* h) {
  if (!h->batch) return BatchPlanOut{};
  const BatchPlan& P = h->batch->plan;
  return BatchPlanOut{P.grid, (int)P.team_size.size(), P.alpha, h->batch->graph_ok ? 1 : 0,
                      {P.floors[0], P.floors[1], P.floors[2], P.floors[3]}};
}

int batch_count(const enkf_handle_s* h) { return h->batch ? h->batch->count : 0; }

size_t batch_state_bytes(const enkf_handle_s* h, int i) {
  const enkf_config& c = h->batch->cfg[i];
  return sizeof(float) * (size_t)c.n * (size_t)c.N;
}

void batch_free(enkf_handle_s* h) {
  BatchState* B = h->batch;
  if (!B) return;
  drop_graph(*B);
  if (B->io_copied) cudaEventDestroy(B->io_copied);
  if (B->h_io) cudaFreeHost(B->h_io);
  void* ptrs[] = {B->arena, B->d_probs, B->d_io, B->d_plan, B->d_status, B->d_bar, B->d_team, B->d_time,
                  B->d_phase};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete B;
  h->batch = nullptr;
}

}  // namespace enkf
