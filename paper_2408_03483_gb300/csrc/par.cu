// Concurrent host tasks over CUDA streams: independent rounds, crosses and
// reciprocals of one stage run side by side so their one-CTA factorisations
// occupy different SMs.
#include <mutex>
#include <thread>
#include <algorithm>

#include "tt_common.cuh"

namespace ttfv {

int sm_count() {
  static std::once_flag once;
  static int n = 152;
  std::call_once(once, [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
  });
  return n;
}


int smem_optin_max() {
  static int v = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 227 * 1024;
  });
  return v;
}

cudaError_t smem_attr_once_impl(const void* fn) {
  static std::mutex mu;
  static std::vector<const void*> done;
  std::lock_guard<std::mutex> lk(mu);
  for (const void* f : done)
    if (f == fn) return cudaSuccess;
  // the dynamic limit plus the kernel's static shared memory may not exceed
  // the opt-in maximum
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  const int dyn = smem_optin_max() - (int)fa.sharedSizeBytes;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  if (e == cudaSuccess) done.push_back(fn);
  return e;
}

cudaStream_t StreamPool::stream(size_t i) {
  while (streams.size() <= i) {
    cudaStream_t s;
    TT_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    streams.push_back(s);
  }
  return streams[i];
}

cudaEvent_t StreamPool::event(size_t i) {
  while (events.size() <= i) {
    cudaEvent_t e;
    TT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    events.push_back(e);
  }
  return events[i];
}

StreamPool::~StreamPool() {
  for (cudaStream_t s : streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : events) cudaEventDestroy(e);
}

static void merge_counters(Exec& dst, const Exec& src) {
  dst.rounds += src.rounds;
  dst.learned_calls += src.learned_calls;
  dst.learned_accepted += src.learned_accepted;
  dst.qb_attempts += src.qb_attempts;
  dst.qb_uncertified += src.qb_uncertified;
  dst.syncs += src.syncs;
  dst.jacobi_sweeps += src.jacobi_sweeps;
  dst.cross_calls += src.cross_calls;
  dst.cross_sweeps += src.cross_sweeps;
  dst.taylor_iters += src.taylor_iters;
  dst.cap_hits += src.cap_hits;
  dst.svd_calls += src.svd_calls;
  dst.svd_p += src.svd_p;
  dst.svd_pd += src.svd_pd;
  dst.svd_sweeps += src.svd_sweeps;
  dst.flops += src.flops;
  dst.bytes += src.bytes;
}

namespace {
struct Child {
  Arena ar;
  Exec ex;
  Prof prof;
  int hi[16];
  double hd[16];
  tt_status err = TT_OK;
};
}  // namespace

void parallel_tasks(Exec& ex, int ntasks, const std::function<void(Exec&, int)>& body) {
  if (ntasks <= 0) return;
  std::vector<Child> ch(ntasks);
  if (ex.dry || ex.pool == nullptr || (ex.prof && ex.prof->on)) {
    // sizing pass, no stream pool, or profiling (per-launch event times must
    // not include queueing behind other streams): tasks in order; the sizing
    // pass gives each task its own arena and reserves the largest footprint
    // once per task
    size_t maxpeak = 0;
    for (int i = 0; i < ntasks; ++i) {
      Child& c = ch[i];
      c.ar.dry = ex.dry;
      c.ex = ex;
      c.ex.ar = ex.dry ? &c.ar : ex.ar;
      c.ex.rounds = c.ex.qb_attempts = c.ex.qb_uncertified = c.ex.syncs = 0;
      c.ex.jacobi_sweeps = c.ex.cross_calls = c.ex.cross_sweeps = c.ex.taylor_iters = c.ex.cap_hits = 0;
      c.ex.svd_calls = c.ex.svd_p = c.ex.svd_pd = c.ex.svd_sweeps = 0;
      c.ex.learned_calls = c.ex.learned_accepted = 0;
      c.ex.flops = c.ex.bytes = 0.0;
      body(c.ex, i);
      merge_counters(ex, c.ex);
      maxpeak = std::max(maxpeak, c.ar.peak);
    }
    if (ex.dry) {
      const size_t need = ex.ar->off + maxpeak * (size_t)ntasks + 256 * (size_t)ntasks;
      if (need > ex.ar->peak) ex.ar->peak = need;
    }
    return;
  }
  Arena& par = *ex.ar;
  const size_t free = par.cap > par.off ? par.cap - par.off : 0;
  const size_t slice = (free / (size_t)ntasks) & ~size_t(255);
  cudaEvent_t start = ex.pool->event(0);
  TT_CUDA(cudaEventRecord(start, ex.s));
  for (int i = 0; i < ntasks; ++i) {
    Child& c = ch[i];
    c.ar.base = par.base + par.off + slice * (size_t)i;
    c.ar.cap = slice;
    c.ex = Exec{};
    c.ex.s = ex.pool->stream((size_t)i);
    c.ex.ar = &c.ar;
    c.ex.dev_status = ex.dev_status;
    c.ex.precision = ex.precision;
    c.ex.pivot_net = ex.pivot_net;
    c.ex.pivot_rec = ex.pivot_rec;
    c.ex.h_pinned = c.hi;
    c.ex.h_pinned_d = c.hd;
    c.prof.on = ex.prof && ex.prof->on;
    c.ex.prof = &c.prof;
    c.ex.pool = nullptr;  // no nesting
    TT_CUDA(cudaStreamWaitEvent(c.ex.s, start, 0));
  }
  std::vector<std::thread> th;
  th.reserve(ntasks);
  for (int i = 0; i < ntasks; ++i) {
    th.emplace_back([&, i] {
      Child& c = ch[i];
      try {
        body(c.ex, i);
      } catch (const Error& e) {
        c.err = e.code;
      } catch (...) {
        c.err = TT_ERR_CUDA;
      }
    });
  }
  for (std::thread& t : th) t.join();
  tt_status first = TT_OK;
  for (int i = 0; i < ntasks; ++i) {
    Child& c = ch[i];
    cudaEvent_t done = ex.pool->event((size_t)i + 1);
    TT_CUDA(cudaEventRecord(done, c.ex.s));
    TT_CUDA(cudaStreamWaitEvent(ex.s, done, 0));
    merge_counters(ex, c.ex);
    if (ex.prof) {
      ex.prof->pending.insert(ex.prof->pending.end(), c.prof.pending.begin(), c.prof.pending.end());
      ex.prof->pool.insert(ex.prof->pool.end(), c.prof.pool.begin(), c.prof.pool.end());
      for (int k = 0; k < K_NCLASS; ++k) {
        ex.prof->ms[k] += c.prof.ms[k];
        ex.prof->flops[k] += c.prof.flops[k];
        ex.prof->bytes[k] += c.prof.bytes[k];
        ex.prof->n[k] += c.prof.n[k];
      }
    }
    if (c.err != TT_OK && first == TT_OK) first = c.err;
  }
  if (first != TT_OK) throw Error{first};
}

}  // namespace ttfv
