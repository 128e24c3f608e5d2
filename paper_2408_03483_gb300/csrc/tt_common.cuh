// Shared declarations of the TT finite-volume CUDA library (sm_103a, FP64 path).
//
// A 2-D TT X[i, j] = sum_k a[k * n1 + i] * b[k * n2 + j]: both cores column-major
// with the mode index fastest (the paper's G1(i) and G2(j)^T, Sec. 3.1).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <functional>
#include <mutex>
#include <vector>

#include "../../include/tt_fv.h"

namespace ttfv {

// ---------------------------------------------------------------- errors
struct Error {
  tt_status code;
};

#define TT_CUDA(call)                                     \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) throw ::ttfv::Error{TT_ERR_CUDA}; \
  } while (0)
#define TT_LAUNCH() TT_CUDA(cudaGetLastError())
#define TT_REQUIRE(cond, code) \
  do {                         \
    if (!(cond)) throw ::ttfv::Error{code}; \
  } while (0)

// Device-side status bits (latched in a device word, read at sync points).
enum : unsigned {
  DEV_JACOBI_NOCONV = 1u,
  DEV_MAXVOL_NOCONV = 2u,
  DEV_SHAPE = 4u,
  DEV_TC_TIMEOUT = 8u,  // a tensor-core kernel gave up waiting on an mbarrier
  DEV_NONFINITE = 16u,  // a small SVD received a NaN/Inf matrix (result zeroed)
};

// ---------------------------------------------------------------- workspace
// Bump allocator over caller-provided device memory (256-byte aligned).
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  size_t peak = 0;
  bool dry = false;  // sizing pass: count only
  template <typename T>
  T* get(size_t n) {
    size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
    size_t o = off;
    off += bytes;
    if (off > peak) peak = off;
    if (dry) return reinterpret_cast<T*>(uintptr_t(0x100) + o);
    if (off > cap) throw Error{TT_ERR_OOM};
    return reinterpret_cast<T*>(base + o);
  }
  size_t mark() const { return off; }
  void reset(size_t m) { off = m; }
};

struct Scope {  // restores the arena on exit
  Arena& a;
  size_t m;
  explicit Scope(Arena& ar) : a(ar), m(ar.mark()) {}
  ~Scope() { a.reset(m); }
};

// ---------------------------------------------------------------- profiling
// Kernel classes for the opt-in per-launch event timing (TT_K_* in the header).
enum KClass : int {
  K_GEMM = TT_K_GEMM,
  K_FORM = TT_K_FORM,
  K_QR = TT_K_QR,
  K_QR_APPLY = TT_K_QR_APPLY,
  K_JACOBI = TT_K_JACOBI,
  K_MAXVOL = TT_K_MAXVOL,
  K_EVAL = TT_K_EVAL,
  K_STENCIL = TT_K_STENCIL,
  K_OTHER = TT_K_OTHER,
  K_QR_MERGE = TT_K_QR_MERGE,
  K_QR_APPLY_MERGE = TT_K_QR_APPLY_MERGE,
  K_NCLASS = TT_K_NCLASS
};
struct Prof {
  bool on = false;
  struct Rec {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double ms[K_NCLASS] = {}, flops[K_NCLASS] = {}, bytes[K_NCLASS] = {};
  long long n[K_NCLASS] = {};
};
extern std::atomic<unsigned long long> g_launches;

// A TT held by the library: device cores with host-known shape and rank.
struct TT {
  int n1 = 0, n2 = 0, r = 0, cap = 0;
  double* a = nullptr;
  double* b = nullptr;
};

// Streams and events for concurrent host tasks (owned by a solver context).
// Also a block of page-locked host slots, one per concurrent task, for the
// small device-to-host reads at sync points (a read into pageable memory goes
// through the driver's staging buffer, which concurrent tasks would share).
struct StreamPool {
  static constexpr size_t kSlots = 64, kSlotBytes = 256;  // int[16] then double[16]
  std::vector<cudaStream_t> streams;
  std::vector<cudaStream_t> streams_hi;  // the device's greatest stream priority
  std::vector<cudaEvent_t> events;
  char* pinned = nullptr;
  bool pinned_failed = false;
  cudaStream_t stream(size_t i);
  cudaStream_t stream_hi(size_t i);
  cudaEvent_t event(size_t i);
  // slot i (< kSlots), or null if page-locked memory is unavailable
  char* slot(size_t i);
  ~StreamPool();
};

// Device parameters of the learned-pivot network (FP32 masters; mlp.cu)
struct MlpNet {
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
};
struct PivotRecorder;  // training-data capture of the crosses (fv.cu)

// Execution context of one call chain.
struct Exec {
  cudaStream_t s = nullptr;
  Arena* ar = nullptr;
  unsigned* dev_status = nullptr;   // device status word
  int* h_pinned = nullptr;          // small pinned host buffer for syncs
  double* h_pinned_d = nullptr;
  bool dry = false;                 // workspace sizing pass: no launches
  int precision = TT_FP64;          // tt_precision of the rounding contractions
  const MlpNet* pivot_net = nullptr;  // learned initial cross pivots (null: maxvol start)
  PivotRecorder* pivot_rec = nullptr; // capture (features, converged pivots) of each cross
  // counters (host)
  long long rounds = 0, qb_attempts = 0, qb_uncertified = 0, syncs = 0;
  long long jacobi_sweeps = 0, cross_calls = 0, cross_sweeps = 0;
  long long taylor_iters = 0, cap_hits = 0;
  int last_rank = 0;  // kept rank of the latest rounding (node trace)
  long long svd_calls = 0, svd_p = 0, svd_pd = 0, svd_sweeps = 0;
  long long learned_calls = 0, learned_accepted = 0;
  long long launches = 0;           // kernels this context launched
  double flops = 0.0, bytes = 0.0;
  Prof* prof = nullptr;             // per-class event timing when prof->on
  StreamPool* pool = nullptr;       // streams for parallel_tasks (null: run tasks in order)
  // range-finder sketch width of the calling site: read as the first
  // sketch's width when larger than the default, set to the certified width
  // (null: default first sketch)
  int* rf_hint = nullptr;
  // TSQR tile shape (tunable): leaf rows as a multiple of max(64, p rounded
  // up to 32), and the largest merge fan-in (0: default).  Two multiples by
  // default: at 4096^2 the step measured 136 ms with single ones, 124 with
  // two, 122 with three and 125 with four (fewer leaves and merge nodes
  // competing for the SMs), the same at 256^2.
  int qr_leaf_mult = 2, qr_fanin = 0;
  // the small SVD may spread its FP64 sweeps over a thread-block cluster: on
  // for the standalone entry points, off in the solver, whose stage runs many
  // roundings at once (the 4096^2 step measured 1.5 % faster with one CTA per
  // SVD: 122.3 / 123.2 against 124.5 / 124.5 ms)
  bool svd_cluster = true;
};

// Wait on the host until ex.s has drained (the sync point of a read-back).
// A stream synchronize: polling an event with a yield measured the same on
// the stage graph (16 to 32 workers), a blocking-sync event 6 % slower.
void host_wait(Exec& ex);

// Run body(child, i) for i < ntasks as concurrent host threads, each on its
// own stream (ordered after ex.s) with its own slice of the free arena; ex.s
// then waits for every task.  Counters and profile records merge into ex.
// Tasks must be independent.  The first task error is rethrown.
void parallel_tasks(Exec& ex, int ntasks, const std::function<void(Exec&, int)>& body);

// Dependency-driven execution of host tasks.  A node is a host function that
// queues GPU work on the stream of the Exec it is given; it runs once every
// node it depends on has run, on one of `workers` host threads, each with its
// own stream and arena slice, and that stream first waits for the GPU work of
// its dependencies.  Nodes may add nodes while the graph runs (loops whose trip
// count is read back from the device); a node added with hold = true also
// waits for release(), and depend() may give it further dependencies until
// then.  Scratch a node takes from its arena is released when it returns, so
// results that outlive a node live in the caller's arena.  Without a stream
// pool, in the sizing pass and when profiling, nodes run one at a time on ex
// in priority order.  run() returns once every node has run and ex.s is
// ordered after their work; it rethrows the first node error.
class TaskGraph {
 public:
  using Fn = std::function<void(Exec&)>;
  TaskGraph(Exec& ex, int workers);
  ~TaskGraph();
  TaskGraph(const TaskGraph&) = delete;
  TaskGraph& operator=(const TaskGraph&) = delete;
  // urgent: queue the node's GPU work on a stream of the device's greatest
  // priority (nodes on the step's longest dependency chain), so that the
  // block scheduler places its CTAs before those of other nodes as SMs free up
  int add(const char* name, int priority, Fn fn, const std::vector<int>& deps = {}, bool hold = false,
          bool urgent = false);
  void depend(int node, int dep);
  void release(int node);
  void run();
  // id of the node the calling thread is running (-1 outside a node)
  static int self();

 private:
  struct Impl;
  Impl* im;
};

// Bracket one kernel launch: counts it, checks the launch, adds its
// algorithmic flops/bytes to the totals and, when profiling, times it.
cudaEvent_t prof_begin(Exec& ex);
void prof_end(Exec& ex, cudaEvent_t a, int cls, double flops, double bytes, const char* what);
void prof_flush(Exec& ex);  // after a stream sync: accumulate finished records
#define TT_KERNEL(ex, cls, flops, bytes, ...)                     \
  do {                                                            \
    cudaEvent_t _tt_a = ::ttfv::prof_begin(ex);                   \
    __VA_ARGS__;                                                  \
    ::ttfv::prof_end(ex, _tt_a, cls, (double)(flops), (double)(bytes), #__VA_ARGS__); \
  } while (0)

// ---------------------------------------------------------------- helpers
// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum,
// once per kernel and process (the attribute is global to the function, so it
// must not be changed per launch while other host threads launch it).
int smem_optin_max();
// multiprocessors of the current device (read once per process)
int sm_count();
cudaError_t smem_attr_once_impl(const void* fn);
template <typename K>
inline void smem_attr_once(K kernel) {
  TT_CUDA(smem_attr_once_impl(reinterpret_cast<const void*>(kernel)));
}
inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

// Copy n ints/doubles from device to the pinned buffer and wait (a sync point).
int fetch_int(Exec& ex, const int* d);
// Reads the small-SVD info triple (k, deflated rank, sweeps) of a p x p SVD,
// accounts it, and returns k; with tail, also its two tail doubles into tl
// (one sync for both).
int fetch_svd_info(Exec& ex, const int* d, int p, const double* tail = nullptr, double* tl = nullptr);
void fetch_doubles(Exec& ex, const double* d, int n, double* out);

// TT_DEBUG_SYNC=1: every launch is waited for, and debug_finite() copies an
// array to the host and throws TT_ERR_NONFINITE (printing `what`) if it holds
// a NaN or Inf.  Both are no-ops otherwise.
bool debug_sync();
void debug_finite(Exec& ex, const double* d, long n, const char* what, int a = 0, int b = 0, int c = 0);
void debug_finite(Exec& ex, const float* d, long n, const char* what, int a = 0, int b = 0, int c = 0);

// ---------------------------------------------------------------- kernels (la.cu)
// The dense kernels are templates on the working precision Real (double for
// the FP64 path, float for the FP32 precision form); la.cu instantiates both.
//
// C[i,j] = alpha * sum_k A(i,k) B(k,j) + beta * C[i,j]; A(i,k) = A[i*ars + k*acs] etc.
template <typename Real>
void gemm(Exec& ex, int M, int N, int K, Real alpha, const Real* A, long ars, long acs, const Real* B, long brs,
          long bcs, Real beta, Real* C, long ldc);
// Y[i,j] = (sum_k A1[i,k]B1[j,k]) * (sum_l A2[i,l]B2[j,l]); FP64 cores
// (column-major), each product accumulated in Real.
template <typename Real>
void form_hadamard_full(Exec& ex, int n1, int n2, const double* A1, int r1, const double* B1, const double* A2,
                        int r2, const double* B2, Real* Y, long ldy);
// sum of squares of an m x n column-major matrix, accumulated in FP64 -> device double
template <typename Real>
void sumsq(Exec& ex, const Real* X, int m, int n, long ld, double* out);

// sum_t X[t] Y[t] over n contiguous FP64 entries -> device double (the
// Frobenius inner product of two equally laid out matrices)
void fdot(Exec& ex, const double* X, const double* Y, long n, double* out);

// Householder TSQR of a tall m x p matrix (p <= 112): row blocks of mb0
// rows factored independently, then a g-ary tree of merges of stacked
// triangular factors (g as many as fit in shared memory); Q is kept implicit.
template <typename Real>
struct QRTreeT {
  int m = 0, p = 0, mb0 = 0, nb0 = 0;
  Real* V0 = nullptr;        // leaf reflectors: nb0 blocks of mb0 x p (top entries on the diagonal)
  Real* tau0 = nullptr;      // nb0 x p
  int g = 2;                 // fan-in of a merge node
  std::vector<int> nin;      // inputs of each merge level (bottom-up)
  std::vector<Real*> Vm;     // per merge level: nodes x g x (p x p) bottom-block reflectors
  std::vector<Real*> vtop;   // per merge level: nodes x p top entries (alpha - beta)
  std::vector<Real*> taum;   // per merge level: nodes x p
  Real* R = nullptr;         // final p x p upper triangle (ld p)
};
using QRTree = QRTreeT<double>;
// (X may be FP64 for an FP32 factorisation: the leaves convert on load.)
template <typename Real, typename Src>
void tsqr(Exec& ex, const Src* X, int m, int p, long ldx, QRTreeT<Real>& t);
// Out (m x k, ld ldo) = Q [C; 0] with C p x k (ld ldc); C and Out may be FP64
// around an FP32 factorisation (converted on load / store).
template <typename Real, typename ZT, typename OT>
void tsqr_apply(Exec& ex, const QRTreeT<Real>& t, const ZT* C, int k, long ldc, OT* Out, long ldo);
// The two factorisations (and the two applications) of a rounding in shared
// launches: same column count p, independent matrices.
template <typename Real, typename Src>
void tsqr2(Exec& ex, const Src* X1, int m1, long ldx1, const Src* X2, int m2, long ldx2, int p, QRTreeT<Real>& t1,
           QRTreeT<Real>& t2);
template <typename Real, typename ZT, typename OT>
void tsqr_apply2(Exec& ex, const QRTreeT<Real>& t1, const ZT* C1, long ldc1, OT* Out1, long ldo1,
                 const QRTreeT<Real>& t2, const ZT* C2, long ldc2, OT* Out2, long ldo2, int k);

// One-sided Jacobi SVD of a square p x p matrix M (ld p, p <= 112).  Writes
// the singular values sorted descending to sig (device, p), U*S (p x p, ld p)
// and V (p x p, ld p) column-sorted alike, and the truncation rank for
// (tol, cap) to *k_out (device).  tail_out[0] = discarded Frobenius norm.
void jacobi_svd(Exec& ex, const double* M, int p, double tol, int cap, double* US, double* V,
                double* sig, int* k_out, double* tail_out);

// Maximum-volume rows of U (n x r, ld n): LU-pivoted start then swaps until
// max|B| <= 1 + delta (ties to the smallest row-major index).  I (device, r).
void maxvol(Exec& ex, const double* U, int n, int r, double delta, int max_iter, int* I);

// Tensor-core contraction (tc_gemm.cu): C (M x N, FP32, ld ldc) = alpha A B +
// beta C with A(i,k) = A[i*ars + k*acs], B(k,j) = B[k*brs + j*bcs], on
// tcgen05 in precision TT_TF32 or TT_BF16; with split, the operands are
// decomposed into tensor-core parts whose products reach FP32 accuracy.
int tc_parts(int precision, bool split);
template <typename Src>
void tc_gemm(Exec& ex, int precision, bool split, int M, int N, int K, float alpha, const Src* A, long ars,
             long acs, const Src* B, long brs, long bcs, float beta, float* C, long ldc);

// Elementwise helpers (ops.cu)
void scaled_copy(Exec& ex, double* dst, const double* src, long n, double alpha);
void fill(Exec& ex, double* dst, long n, double v);
// dst (reps n x r, column-major) = src (n x r) repeated reps times down each
// column: dst[c (reps n) + m n + i] = src[c n + i]
void repeat_rows(Exec& ex, double* dst, const double* src, int n, int r, int reps);

}  // namespace ttfv
