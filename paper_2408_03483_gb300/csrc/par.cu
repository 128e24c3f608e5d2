// Concurrent host tasks over CUDA streams: independent rounds, crosses and
// reciprocals of one stage run side by side so their one-CTA factorisations
// occupy different SMs.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <mutex>
#include <queue>
#include <thread>

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

cudaStream_t StreamPool::stream_hi(size_t i) {
  while (streams_hi.size() <= i) {
    int least = 0, greatest = 0;
    TT_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    cudaStream_t s;
    TT_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, greatest));
    streams_hi.push_back(s);
  }
  return streams_hi[i];
}

cudaEvent_t StreamPool::event(size_t i) {
  while (events.size() <= i) {
    cudaEvent_t e;
    TT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    events.push_back(e);
  }
  return events[i];
}

char* StreamPool::slot(size_t i) {
  if (i >= kSlots || pinned_failed) return nullptr;
  if (!pinned) {
    if (cudaHostAlloc(reinterpret_cast<void**>(&pinned), kSlots * kSlotBytes, cudaHostAllocPortable) !=
        cudaSuccess) {
      cudaGetLastError();
      pinned = nullptr;
      pinned_failed = true;
      return nullptr;
    }
  }
  return pinned + i * kSlotBytes;
}

void host_wait(Exec& ex) { TT_CUDA(cudaStreamSynchronize(ex.s)); }

StreamPool::~StreamPool() {
  for (cudaStream_t s : streams) cudaStreamDestroy(s);
  for (cudaStream_t s : streams_hi) cudaStreamDestroy(s);
  for (cudaEvent_t e : events) cudaEventDestroy(e);
  if (pinned) cudaFreeHost(pinned);
}


static void merge_counters(Exec& dst, const Exec& src) {
  dst.rounds += src.rounds;
  dst.learned_calls += src.learned_calls;
  dst.learned_accepted += src.learned_accepted;
  dst.launches += src.launches;
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

static void zero_counters(Exec& e) {
  e.rounds = e.qb_attempts = e.qb_uncertified = e.syncs = 0;
  e.jacobi_sweeps = e.cross_calls = e.cross_sweeps = e.taylor_iters = e.cap_hits = 0;
  e.svd_calls = e.svd_p = e.svd_pd = e.svd_sweeps = 0;
  e.learned_calls = e.learned_accepted = e.launches = 0;
  e.flops = e.bytes = 0.0;
}

// A child context on stream s over arena a, sharing the parent's device status
// word, precision, pivot network and recorder; no stream pool (no nesting).
static void child_exec(const Exec& parent, Exec& c, Arena* a, cudaStream_t s, Prof* prof, int* hi, double* hd,
                       size_t slot) {
  if (char* p = parent.pool ? parent.pool->slot(slot) : nullptr) {
    hi = reinterpret_cast<int*>(p);
    hd = reinterpret_cast<double*>(p + 64);
  }
  c = Exec{};
  c.s = s;
  c.ar = a;
  c.dev_status = parent.dev_status;
  c.precision = parent.precision;
  c.qr_leaf_mult = parent.qr_leaf_mult;
  c.qr_fanin = parent.qr_fanin;
  c.svd_cluster = parent.svd_cluster;
  c.pivot_net = parent.pivot_net;
  c.pivot_rec = parent.pivot_rec;
  c.h_pinned = hi;
  c.h_pinned_d = hd;
  prof->on = parent.prof && parent.prof->on;
  c.prof = prof;
  c.pool = nullptr;
}

static void merge_prof(Exec& ex, const Prof& p) {
  if (!ex.prof) return;
  ex.prof->pending.insert(ex.prof->pending.end(), p.pending.begin(), p.pending.end());
  ex.prof->pool.insert(ex.prof->pool.end(), p.pool.begin(), p.pool.end());
  for (int k = 0; k < K_NCLASS; ++k) {
    ex.prof->ms[k] += p.ms[k];
    ex.prof->flops[k] += p.flops[k];
    ex.prof->bytes[k] += p.bytes[k];
    ex.prof->n[k] += p.n[k];
  }
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
      zero_counters(c.ex);
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
    child_exec(ex, c.ex, &c.ar, ex.pool->stream((size_t)i), &c.prof, c.hi, c.hd, (size_t)i + 1);
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
    merge_prof(ex, c.prof);
    if (c.err != TT_OK && first == TT_OK) first = c.err;
  }
  if (first != TT_OK) throw Error{first};
}

// ---------------------------------------------------------------- task graph
namespace {
struct GNode {
  const char* name = "";
  int prio = 0;
  bool urgent = false;  // GPU work on the worker's high-priority stream
  TaskGraph::Fn fn;
  std::vector<int> in;   // every dependency (the GPU-side waits)
  std::vector<int> out;  // dependents still counting on this node
  int pending = 0;       // unfinished dependencies, plus one while held
  bool done = false;
  cudaEvent_t ev = nullptr;
};

struct GWorker {
  Arena ar;
  Exec ex;
  Prof prof;
  int hi[16];
  double hd[16];
};

struct TraceRec {
  const char* name;
  int worker;
  double t0, t1;  // microseconds from the start of run()
  // the node's own work: host syncs, range-finder attempts, small SVDs and
  // the sum of their sizes, cross sweeps, kernel launches
  long long syncs, qb, svd, svd_p, sweeps, launches;
  int rank;  // kept rank of the worker's latest rounding
};

struct Tally {
  long long syncs, qb, svd, svd_p, sweeps, launches;
  explicit Tally(const Exec& e)
      : syncs(e.syncs), qb(e.qb_attempts), svd(e.svd_calls), svd_p(e.svd_p), sweeps(e.cross_sweeps),
        launches(e.launches) {}
};

// Events of graph nodes are taken from the stream pool above those that
// parallel_tasks uses (one per task plus the start event); a worker that
// moves between its two streams orders them by event kSwitchEvent0 + worker.
constexpr size_t kSwitchEvent0 = 32;
constexpr size_t kGraphEvent0 = 64;

// TT_STREAM_PRIORITY=0 (environment, read once) queues urgent nodes on the
// ordinary streams too, for comparison.
bool stream_priority_on() {
  static const bool v = [] {
    const char* e = std::getenv("TT_STREAM_PRIORITY");
    return !(e && e[0] == '0');
  }();
  return v;
}

thread_local int t_self = -1;

// Runs fn as node id on this thread (TaskGraph::self() answers id meanwhile).
struct SelfScope {
  int saved;
  explicit SelfScope(int id) : saved(t_self) { t_self = id; }
  ~SelfScope() { t_self = saved; }
};

const char* trace_path() {
  static const char* p = std::getenv("TT_TRACE");
  return (p && *p) ? p : nullptr;
}
}  // namespace

struct TaskGraph::Impl {
  Exec& ex;
  int workers;
  bool serial;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<GNode> nodes;
  std::priority_queue<std::pair<int, int>> ready;  // (priority, -id): high priority, then oldest
  int remaining = 0;  // nodes not yet finished (held ones included)
  int running = 0;
  tt_status err = TT_OK;
  std::vector<TraceRec> trace;
  std::chrono::steady_clock::time_point t_start;

  Impl(Exec& e, int w)
      : ex(e), workers(std::max(1, w)), serial(e.dry || e.pool == nullptr || (e.prof && e.prof->on)) {}

  double now_us() const {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t_start).count();
  }
  void push_ready(int id) {
    ready.push({nodes[id].prio, -id});
    cv.notify_one();
  }
  // under mu
  void finish(int id, tt_status st, int worker, double t0, const Tally& before, const Exec& after) {
    GNode& n = nodes[id];
    n.done = true;
    --remaining;
    --running;
    for (int o : n.out)
      if (--nodes[o].pending == 0) push_ready(o);
    n.out.clear();
    if (st != TT_OK && err == TT_OK) err = st;
    if (trace_path())
      trace.push_back(TraceRec{n.name, worker, t0, now_us(), after.syncs - before.syncs,
                               after.qb_attempts - before.qb, after.svd_calls - before.svd,
                               after.svd_p - before.svd_p, after.cross_sweeps - before.sweeps,
                               after.launches - before.launches, after.last_rank});
    cv.notify_all();
  }
  void write_trace() {
    static std::mutex fmu;
    static long long graph_seq = 0;
    std::lock_guard<std::mutex> lk(fmu);
    FILE* f = std::fopen(trace_path(), "a");
    if (!f) return;
    const long long g = graph_seq++;
    for (const TraceRec& r : trace)
      std::fprintf(f,
                   "{\"graph\": %lld, \"name\": \"%s\", \"worker\": %d, \"t0_us\": %.1f, \"t1_us\": %.1f, "
                   "\"syncs\": %lld, \"qb\": %lld, \"svd\": %lld, \"svd_p\": %lld, \"sweeps\": %lld, "
                   "\"launches\": %lld, \"rank\": %d}\n",
                   g, r.name, r.worker, r.t0, r.t1, r.syncs, r.qb, r.svd, r.svd_p, r.sweeps, r.launches, r.rank);
    std::fclose(f);
  }
  void run_serial();
  void run_parallel();
};

TaskGraph::TaskGraph(Exec& ex, int workers) : im(new Impl(ex, workers)) {}
TaskGraph::~TaskGraph() { delete im; }
int TaskGraph::self() { return t_self; }

int TaskGraph::add(const char* name, int priority, Fn fn, const std::vector<int>& deps, bool hold, bool urgent) {
  std::lock_guard<std::mutex> lk(im->mu);
  const int id = (int)im->nodes.size();
  for (int d : deps) TT_REQUIRE(d < id, TT_ERR_ARG);
  im->nodes.emplace_back();
  GNode& n = im->nodes.back();
  n.name = name;
  n.prio = priority;
  n.urgent = urgent;
  n.fn = std::move(fn);
  n.pending = hold ? 1 : 0;
  for (int d : deps) {
    if (d < 0) continue;  // "no node": lets callers pass optional dependencies
    n.in.push_back(d);
    if (!im->nodes[d].done) {
      im->nodes[d].out.push_back(id);
      n.pending++;
    }
  }
  if (!im->serial) n.ev = im->ex.pool->event(kGraphEvent0 + (size_t)id);
  im->remaining++;
  if (n.pending == 0) im->push_ready(id);
  return id;
}

void TaskGraph::depend(int node, int dep) {
  std::lock_guard<std::mutex> lk(im->mu);
  TT_REQUIRE(node >= 0 && node < (int)im->nodes.size() && dep < (int)im->nodes.size(), TT_ERR_ARG);
  GNode& n = im->nodes[node];
  TT_REQUIRE(n.pending > 0 && !n.done, TT_ERR_ARG);  // only a held node takes new dependencies
  if (dep < 0) return;
  n.in.push_back(dep);
  if (!im->nodes[dep].done) {
    im->nodes[dep].out.push_back(node);
    n.pending++;
  }
}

void TaskGraph::release(int node) {
  std::lock_guard<std::mutex> lk(im->mu);
  TT_REQUIRE(node >= 0 && node < (int)im->nodes.size(), TT_ERR_ARG);
  GNode& n = im->nodes[node];
  TT_REQUIRE(n.pending > 0 && !n.done, TT_ERR_ARG);
  if (--n.pending == 0) im->push_ready(node);
}

void TaskGraph::Impl::run_serial() {
  size_t maxpeak = 0;
  for (;;) {
    int id;
    Fn fn;
    double t0;
    {
      std::lock_guard<std::mutex> lk(mu);
      if (ready.empty()) break;
      id = -ready.top().second;
      ready.pop();
      running++;
      fn = std::move(nodes[id].fn);
      t0 = now_us();
    }
    if (ex.dry) {
      // sizing pass: each node on an arena of its own; the parallel run gives
      // every worker a slice of the largest footprint
      Arena a;
      a.dry = true;
      Exec e = ex;
      e.ar = &a;
      zero_counters(e);
      SelfScope me(id);
      fn(e);
      merge_counters(ex, e);
      maxpeak = std::max(maxpeak, a.peak);
      std::lock_guard<std::mutex> lk(mu);
      finish(id, TT_OK, 0, t0, Tally(ex), ex);
      continue;
    }
    const Tally before(ex);
    {
      Scope sc(*ex.ar);
      SelfScope me(id);
      fn(ex);
    }
    std::lock_guard<std::mutex> lk(mu);
    finish(id, TT_OK, 0, t0, before, ex);
  }
  TT_REQUIRE(remaining == 0, TT_ERR_ARG);  // a held node was never released
  if (ex.dry) {
    const size_t need = ex.ar->off + (maxpeak + 256) * (size_t)workers;
    if (need > ex.ar->peak) ex.ar->peak = need;
  }
}

void TaskGraph::Impl::run_parallel() {
  Arena& par = *ex.ar;
  const size_t free = par.cap > par.off ? par.cap - par.off : 0;
  const size_t slice = (free / (size_t)workers) & ~size_t(255);
  std::vector<GWorker> wk(workers);
  cudaEvent_t start = ex.pool->event(0);
  TT_CUDA(cudaEventRecord(start, ex.s));
  for (int i = 0; i < workers; ++i) {
    GWorker& w = wk[i];
    w.ar.base = par.base + par.off + slice * (size_t)i;
    w.ar.cap = slice;
    child_exec(ex, w.ex, &w.ar, ex.pool->stream((size_t)i), &w.prof, w.hi, w.hd, (size_t)i + 1);
    TT_CUDA(cudaStreamWaitEvent(w.ex.s, start, 0));
  }
  const bool prio = stream_priority_on() && workers <= int(kGraphEvent0 - kSwitchEvent0);
  // created here: the pool's vectors are not touched by the worker threads
  std::vector<cudaStream_t> s_hi(workers, nullptr);
  std::vector<cudaEvent_t> s_sw(workers, nullptr);
  if (prio)
    for (int i = 0; i < workers; ++i) {
      s_hi[i] = ex.pool->stream_hi((size_t)i);
      s_sw[i] = ex.pool->event(kSwitchEvent0 + (size_t)i);
    }
  auto loop = [&](int wi) {
    GWorker& w = wk[wi];
    cudaStream_t s_lo = w.ex.s;
    std::vector<cudaEvent_t> waits;
    for (;;) {
      int id;
      Fn fn;
      cudaEvent_t ev;
      double t0;
      bool urg;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return !ready.empty() || err != TT_OK || remaining == 0 || running == 0; });
        if (err != TT_OK || remaining == 0) return;
        if (ready.empty()) {  // nothing runs and nothing is ready: a held node was never released
          err = TT_ERR_ARG;
          cv.notify_all();
          return;
        }
        id = -ready.top().second;
        ready.pop();
        running++;
        GNode& n = nodes[id];
        fn = std::move(n.fn);
        ev = n.ev;
        urg = prio && n.urgent;
        waits.clear();
        for (int d : n.in) waits.push_back(nodes[d].ev);
        t0 = now_us();
      }
      tt_status st = TT_OK;
      const Tally before(w.ex);
      try {
        // the worker's two streams share its arena slice: the stream taken
        // next waits for everything queued on the other one
        const cudaStream_t want = urg ? s_hi[wi] : s_lo;
        if (want != w.ex.s) {
          TT_CUDA(cudaEventRecord(s_sw[wi], w.ex.s));
          TT_CUDA(cudaStreamWaitEvent(want, s_sw[wi], 0));
          w.ex.s = want;
        }
        for (cudaEvent_t e : waits) TT_CUDA(cudaStreamWaitEvent(w.ex.s, e, 0));
        Scope sc(w.ar);
        SelfScope me(id);
        fn(w.ex);
        TT_CUDA(cudaEventRecord(ev, w.ex.s));
      } catch (const Error& e) {
        st = e.code;
      } catch (...) {
        st = TT_ERR_CUDA;
      }
      std::lock_guard<std::mutex> lk(mu);
      finish(id, st, wi, t0, before, w.ex);
    }
  };
  std::vector<std::thread> th;
  th.reserve(workers);
  for (int i = 0; i < workers; ++i) th.emplace_back(loop, i);
  for (std::thread& t : th) t.join();
  for (int i = 0; i < workers; ++i) {
    GWorker& w = wk[i];
    cudaEvent_t done = ex.pool->event((size_t)i + 1);
    TT_CUDA(cudaEventRecord(done, w.ex.s));
    TT_CUDA(cudaStreamWaitEvent(ex.s, done, 0));
    merge_counters(ex, w.ex);
    merge_prof(ex, w.prof);
  }
  if (err != TT_OK) throw Error{err};
}

void TaskGraph::run() {
  im->t_start = std::chrono::steady_clock::now();
  if (im->serial)
    im->run_serial();
  else
    im->run_parallel();
  if (trace_path() && !im->ex.dry) im->write_trace();
}

}  // namespace ttfv
