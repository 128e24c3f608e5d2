// Ensemble driver (batched form): many independent solver instances of uneven
// grid size, rank cap and reconstruction advanced together on one GPU.
//
// Each instance owns a stream and a slice of one caller workspace.  A batch
// step advances every instance by one SSP-RK3 step: a pool of host workers
// takes instances from a shared queue in longest-first order (the cost of an
// instance is the wall time of its previous step), so the GPU sees the
// kernels of `workers` instances at once -- the single-instance path leaves
// most SMs idle between its rank-dependent launches.  The worker count and
// whether each instance also runs its own independent stage tasks
// concurrently are tunables; tt_fv_batch_tune times candidates on real
// steps and keeps the fastest.  tt_fv_batch_tune_tiles picks each instance's
// TSQR tile shape (leaf rows, merge fan-in) from the same kind of trials.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <numeric>
#include <thread>
#include <vector>

#include "tt_common.cuh"

namespace ttfv {
void solver_task_pool(tt_fv_ctx* ctx, bool on);  // fv.cu
}  // namespace ttfv

using namespace ttfv;

struct tt_fv_batch {
  std::vector<tt_fv_ctx*> inst;
  std::vector<cudaStream_t> streams;
  std::vector<double> cost;  // seconds of each instance's last step
  std::vector<long long> cells;
  int workers = 8;
  bool inner_tasks = false;
  cudaStream_t user = nullptr;
  cudaEvent_t ev = nullptr;
};

namespace {

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

void release(tt_fv_batch* b) {
  for (tt_fv_ctx* c : b->inst)
    if (c) tt_fv_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->ev) cudaEventDestroy(b->ev);
  delete b;
}

// One batch step over all instances with the current configuration.
tt_status batch_step(tt_fv_batch* b) {
  const int n = (int)b->inst.size();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  std::atomic<int> next{0};
  std::atomic<int> err{TT_OK};
  auto work = [&] {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n || err.load() != TT_OK) return;
      const int i = order[k];
      const auto t0 = std::chrono::steady_clock::now();
      tt_status r = tt_fv_step(b->inst[i], 1);
      if (r == TT_OK && cudaStreamSynchronize(b->streams[i]) != cudaSuccess) r = TT_ERR_CUDA;
      b->cost[i] = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (r != TT_OK) {
        int expect = TT_OK;
        err.compare_exchange_strong(expect, r);
        return;
      }
    }
  };
  const int w = std::max(1, std::min(b->workers, n));
  std::vector<std::thread> th;
  th.reserve(w);
  for (int t = 0; t < w; ++t) th.emplace_back(work);
  for (std::thread& t : th) t.join();
  if (err.load() != TT_OK) return (tt_status)err.load();
  // the caller's stream is ordered after every instance's work
  for (int i = 0; i < n; ++i) {
    if (cudaEventRecord(b->ev, b->streams[i]) != cudaSuccess) return TT_ERR_CUDA;
    if (cudaStreamWaitEvent(b->user, b->ev, 0) != cudaSuccess) return TT_ERR_CUDA;
  }
  return TT_OK;
}

}  // namespace

extern "C" {

size_t tt_fv_batch_workspace_size(const tt_fv_params* p, int32_t count) {
  if (!p || count < 1) return 0;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const size_t s = tt_fv_workspace_size(&p[i]);
    if (s == 0) return 0;
    total += align256(s);
  }
  return total;
}

tt_status tt_fv_batch_init(const tt_fv_params* p, int32_t count, const tt2* q0, void* ws, size_t ws_bytes,
                           void* stream, tt_fv_batch** out) {
  if (!p || count < 1 || !q0 || !ws || !out) return TT_ERR_ARG;
  tt_fv_batch* b = new (std::nothrow) tt_fv_batch();
  if (!b) return TT_ERR_OOM;
  b->user = static_cast<cudaStream_t>(stream);
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    release(b);
    return TT_ERR_CUDA;
  }
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    const size_t need = tt_fv_workspace_size(&p[i]);
    if (need == 0) {
      release(b);
      return TT_ERR_ARG;
    }
    if (off + need > ws_bytes) {
      release(b);
      return TT_ERR_OOM;
    }
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      release(b);
      return TT_ERR_CUDA;
    }
    b->streams.push_back(s);
    // the instance's first work (tt_fv_init copies q0) follows whatever the
    // caller queued on its stream, e.g. the writes of q0 itself
    if (cudaEventRecord(b->ev, b->user) != cudaSuccess || cudaStreamWaitEvent(s, b->ev, 0) != cudaSuccess) {
      release(b);
      return TT_ERR_CUDA;
    }
    tt_fv_ctx* c = nullptr;
    const tt_status r = tt_fv_init(&p[i], &q0[3 * i], static_cast<char*>(ws) + off, need, s, &c);
    if (r != TT_OK) {
      release(b);
      return r;
    }
    b->inst.push_back(c);
    solver_task_pool(c, b->inner_tasks);
    off += align256(need);
    const long long cells = (long long)p[i].nx * p[i].ny;
    b->cells.push_back(cells);
    // first-step order: cells x rank cap^2 as the cost estimate
    b->cost.push_back(1e-12 * (double)cells * p[i].rank_cap * p[i].rank_cap);
  }
  *out = b;
  return TT_OK;
}

tt_status tt_fv_batch_configure(tt_fv_batch* b, int32_t workers, int32_t inner_tasks) {
  if (!b || workers < 1) return TT_ERR_ARG;
  b->workers = workers;
  b->inner_tasks = inner_tasks != 0;
  for (tt_fv_ctx* c : b->inst) solver_task_pool(c, b->inner_tasks);
  return TT_OK;
}

tt_status tt_fv_batch_step(tt_fv_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return TT_ERR_ARG;
  for (int s = 0; s < nsteps; ++s) {
    const tt_status r = batch_step(b);
    if (r != TT_OK) return r;
  }
  return TT_OK;
}

tt_status tt_fv_batch_tune(tt_fv_batch* b, const int32_t* workers, int32_t ncand, int32_t steps_per_trial,
                           int32_t* best_workers, int32_t* best_inner, double* rates) {
  if (!b || !workers || ncand < 1 || steps_per_trial < 1) return TT_ERR_ARG;
  const double cells = (double)std::accumulate(b->cells.begin(), b->cells.end(), 0LL);
  double best = -1.0;
  int bw = b->workers;
  bool bi = b->inner_tasks;
  for (int c = 0; c < ncand; ++c)
    for (int inner = 0; inner < 2; ++inner) {
      if (workers[c] < 1) return TT_ERR_ARG;
      tt_status r = tt_fv_batch_configure(b, workers[c], inner);
      if (r != TT_OK) return r;
      const auto t0 = std::chrono::steady_clock::now();
      r = tt_fv_batch_step(b, steps_per_trial);
      if (r != TT_OK) return r;
      if (cudaStreamSynchronize(b->user) != cudaSuccess) return TT_ERR_CUDA;
      const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      const double rate = cells * steps_per_trial / std::max(sec, 1e-9);
      if (rates) rates[2 * c + inner] = rate;
      if (rate > best) {
        best = rate;
        bw = workers[c];
        bi = inner != 0;
      }
    }
  const tt_status r = tt_fv_batch_configure(b, bw, bi ? 1 : 0);
  if (best_workers) *best_workers = bw;
  if (best_inner) *best_inner = bi ? 1 : 0;
  return r;
}

tt_status tt_fv_batch_tune_tiles(tt_fv_batch* b, int32_t steps_per_trial, int32_t rounds, int32_t* shape_out,
                                 double* rates) {
  if (!b || steps_per_trial < 1 || rounds < 1) return TT_ERR_ARG;
  const int K = tt_tile_shapes(nullptr, nullptr, 0), n = (int)b->inst.size();
  const double cells = (double)std::accumulate(b->cells.begin(), b->cells.end(), 0LL);
  // the rounds interleave the shapes, so that the ranks' growth over the
  // trial steps does not favour the shapes timed first
  std::vector<double> cost((size_t)n * K, 0.0), sec(K, 0.0);
  for (int r = 0; r < rounds; ++r)
    for (int k = 0; k < K; ++k) {
      for (tt_fv_ctx* c : b->inst) {
        const tt_status e = tt_fv_set_tile_shape(c, k);
        if (e != TT_OK) return e;
      }
      const auto t0 = std::chrono::steady_clock::now();
      for (int st = 0; st < steps_per_trial; ++st) {
        const tt_status e = batch_step(b);
        if (e != TT_OK) return e;
        for (int i = 0; i < n; ++i) cost[(size_t)i * K + k] += b->cost[i];
      }
      if (cudaStreamSynchronize(b->user) != cudaSuccess) return TT_ERR_CUDA;
      sec[k] += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
  if (rates)
    for (int k = 0; k < K; ++k) rates[k] = cells * steps_per_trial * rounds / std::max(sec[k], 1e-9);
  for (int i = 0; i < n; ++i) {
    int best = 0;
    for (int k = 1; k < K; ++k)
      if (cost[(size_t)i * K + k] < cost[(size_t)i * K + best]) best = k;
    const tt_status e = tt_fv_set_tile_shape(b->inst[i], best);
    if (e != TT_OK) return e;
    if (shape_out) shape_out[i] = best;
  }
  return TT_OK;
}

tt_status tt_fv_batch_get(tt_fv_batch* b, int32_t i, tt2 q_out[3]) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return TT_ERR_ARG;
  return tt_fv_get(b->inst[i], q_out);
}

tt_status tt_fv_batch_stats_get(tt_fv_batch* b, int32_t i, tt_fv_stats* out) {
  if (!b || i < 0 || i >= (int)b->inst.size()) return TT_ERR_ARG;
  return tt_fv_stats_get(b->inst[i], out);
}

void tt_fv_batch_destroy(tt_fv_batch* b) {
  if (!b) return;
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  release(b);
}

}  // extern "C"
