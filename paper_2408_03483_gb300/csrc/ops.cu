// TT operations on device cores: periodic core stencils (Sec. 4.3.1 and the
// (T - 1)/dx flux difference of Eq. SWE-system-TT), Gauss-point block sums,
// TT sums by core concatenation, Khatri-Rao Hadamard cores, and TT rounding
// (Sec. 3.2) by three exact routes chosen from the shape.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>

#include <vector>

#include "tt_ops.cuh"

namespace ttfv {

// ============================================================== elementwise
__global__ void k_scaled_copy(double* __restrict__ dst, const double* __restrict__ src, long n, double a) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    dst[t] = a * src[t];
}
__global__ void k_repeat_rows(double* __restrict__ dst, const double* __restrict__ src, int n, int r, int reps) {
  const long per = (long)n * reps, total = per * r;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const long c = t / per;
    dst[t] = src[c * n + (t - c * per) % n];
  }
}
__global__ void k_fill(double* __restrict__ dst, long n, double v) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) dst[t] = v;
}

static int grid_for(long n) { return std::max(1, std::min(ceil_div(n, 256), 1184)); }

void scaled_copy(Exec& ex, double* dst, const double* src, long n, double alpha) {
  if (n <= 0 || ex.dry) return;
  TT_KERNEL(ex, K_OTHER, n, 16.0 * n, k_scaled_copy<<<grid_for(n), 256, 0, ex.s>>>(dst, src, n, alpha));
}
void repeat_rows(Exec& ex, double* dst, const double* src, int n, int r, int reps) {
  const long total = (long)n * reps * r;
  if (total <= 0 || ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 0, 8.0 * (total + (double)n * r),
            k_repeat_rows<<<grid_for(total), 256, 0, ex.s>>>(dst, src, n, r, reps));
}
void fill(Exec& ex, double* dst, long n, double v) {
  if (n <= 0 || ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 0, 8.0 * n, k_fill<<<grid_for(n), 256, 0, ex.s>>>(dst, n, v));
}

// ============================================================== launch accounting
std::atomic<unsigned long long> g_launches{0};

cudaEvent_t prof_begin(Exec& ex) {
  if (!ex.prof || !ex.prof->on) return nullptr;
  Prof& pf = *ex.prof;
  cudaEvent_t a;
  if (!pf.pool.empty()) {
    a = pf.pool.back();
    pf.pool.pop_back();
  } else {
    TT_CUDA(cudaEventCreate(&a));
  }
  TT_CUDA(cudaEventRecord(a, ex.s));
  return a;
}

// TT_DEBUG_SYNC=1 in the environment: wait for every kernel and report the
// first one that fails (its launch expression and index) on stderr.
bool debug_sync() {
  static const bool on = [] {
    const char* v = std::getenv("TT_DEBUG_SYNC");
    return v && v[0] && v[0] != '0';
  }();
  return on;
}

void prof_end(Exec& ex, cudaEvent_t a, int cls, double flops, double bytes, const char* what) {
  const unsigned long long idx = g_launches.fetch_add(1, std::memory_order_relaxed);
  ex.launches++;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && debug_sync()) e = cudaStreamSynchronize(ex.s);
  if (e != cudaSuccess) {
    if (debug_sync())
      std::fprintf(stderr, "tt_fv: launch %llu (class %d) failed: %s\n  %s\n", idx, cls, cudaGetErrorString(e), what);
    throw Error{TT_ERR_CUDA};
  }
  ex.flops += flops;
  ex.bytes += bytes;
  if (!a) return;
  Prof& pf = *ex.prof;
  cudaEvent_t b;
  if (!pf.pool.empty()) {
    b = pf.pool.back();
    pf.pool.pop_back();
  } else {
    TT_CUDA(cudaEventCreate(&b));
  }
  TT_CUDA(cudaEventRecord(b, ex.s));
  pf.pending.push_back(Prof::Rec{cls, a, b, flops, bytes});
}

void prof_flush(Exec& ex) {
  if (!ex.prof || ex.prof->pending.empty()) return;
  Prof& pf = *ex.prof;
  for (const Prof::Rec& r : pf.pending) {
    float ms = 0.0f;
    TT_CUDA(cudaEventSynchronize(r.b));
    TT_CUDA(cudaEventElapsedTime(&ms, r.a, r.b));
    pf.ms[r.cls] += ms;
    pf.flops[r.cls] += r.flops;
    pf.bytes[r.cls] += r.bytes;
    pf.n[r.cls] += 1;
    pf.pool.push_back(r.a);
    pf.pool.push_back(r.b);
  }
  pf.pending.clear();
}

template <typename T>
static void debug_finite_t(Exec& ex, const T* d, long n, const char* what, int a, int b, int c) {
  if (!debug_sync() || ex.dry || n <= 0) return;
  std::vector<T> h((size_t)n);
  TT_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(T) * n, cudaMemcpyDeviceToHost, ex.s));
  TT_CUDA(cudaStreamSynchronize(ex.s));
  for (long i = 0; i < n; ++i)
    if (!std::isfinite((double)h[i])) {
      std::fprintf(stderr, "tt_fv: non-finite %s (%d, %d, %d) at entry %ld of %ld: %g\n", what, a, b, c, i, n,
                   (double)h[i]);
      throw Error{TT_ERR_NONFINITE};
    }
}
void debug_finite(Exec& ex, const double* d, long n, const char* what, int a, int b, int c) {
  debug_finite_t(ex, d, n, what, a, b, c);
}
void debug_finite(Exec& ex, const float* d, long n, const char* what, int a, int b, int c) {
  debug_finite_t(ex, d, n, what, a, b, c);
}

// ============================================================== core stencils
// out_o[i, k] = sum_t c_{o,t} * in[base_{o,t} + (i + s_{o,t}) mod n, k]
// for the n rows of output o; one launch produces every output.
__global__ void k_stencil(StencilSet st, const double* __restrict__ in, long ldin, int n, int r) {
  const int o = blockIdx.z;
  const StencilOut& so = st.out[o];
  for (int k = blockIdx.y; k < r; k += gridDim.y) {
    const double* col = in + (size_t)k * ldin;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double acc = 0.0;
      for (int t = 0; t < so.ntaps; ++t) {
        // periodic wrap without a division: |shift| < n for every stencil
        int ii = i + so.shift[t];
        ii += ii < 0 ? n : 0;
        ii -= ii >= n ? n : 0;
        acc = fma(so.coef[t], col[so.base[t] + ii], acc);
      }
      so.dst[(size_t)so.row0 + i + (size_t)k * so.ld] = acc;
    }
  }
}

void stencil(Exec& ex, const StencilSet& st, const double* in, long ldin, int n, int r) {
  if (r <= 0 || n <= 0) return;
  int taps = 0;
  for (int o = 0; o < st.nout; ++o) {
    taps += st.out[o].ntaps;
    for (int t = 0; t < st.out[o].ntaps; ++t) TT_REQUIRE(std::abs(st.out[o].shift[t]) < n, TT_ERR_ARG);
  }
  if (ex.dry) return;
  TT_REQUIRE(st.nout >= 1 && st.nout <= kMaxStencilOut, TT_ERR_ARG);
  dim3 grid(ceil_div(n, 256), std::min(r, 1024), st.nout);
  // algorithmic bytes: each input column read once, each output written once
  // (a stacked input of several blocks is read block by block)
  int maxbase = 0;
  for (int o = 0; o < st.nout; ++o)
    for (int t = 0; t < st.out[o].ntaps; ++t) maxbase = std::max(maxbase, st.out[o].base[t]);
  const double in_rows = (double)n * (1 + maxbase / std::max(n, 1));
  TT_KERNEL(ex, K_STENCIL, 2.0 * n * (double)r * taps, 8.0 * r * (in_rows + (double)n * st.nout),
            k_stencil<<<grid, 256, 0, ex.s>>>(st, in, ldin, n, r));
}

// ============================================================== Khatri-Rao cores
// Z[i, a*r2 + b] = X[i, a] * Y[i, b] (row-wise Kronecker; the TT Hadamard cores)
__global__ void k_khatri_rao(const double* __restrict__ X, int r1, const double* __restrict__ Y, int r2, int n,
                             double* __restrict__ Z) {
  const long total = (long)n * r1 * r2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = int(t % n);
    const long c = t / n;
    const int a = int(c / r2), b = int(c % r2);
    Z[t] = X[i + (size_t)a * n] * Y[i + (size_t)b * n];
  }
}

// The same with two rows per thread as double2 (n even, 16-byte aligned
// cores): X(i, a) is read once per row pair and kept in registers across the
// r2 output columns a r2 .. a r2 + r2 - 1 (grid y = a); the write-bound part
// is one coalesced 16-byte store per thread and column.
__global__ void k_khatri_rao2(const double* __restrict__ X, int r1, const double* __restrict__ Y, int r2, int n,
                              double* __restrict__ Z) {
  const int h = n >> 1;
  const int a = blockIdx.y;
  const double2* X2 = reinterpret_cast<const double2*>(X + (size_t)a * n);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < h; q += gridDim.x * blockDim.x) {
    const double2 x = X2[q];
    for (int b = 0; b < r2; ++b) {
      const double2 y = reinterpret_cast<const double2*>(Y + (size_t)b * n)[q];
      reinterpret_cast<double2*>(Z + ((size_t)a * r2 + b) * n)[q] = make_double2(x.x * y.x, x.y * y.y);
    }
  }
}

void khatri_rao(Exec& ex, const double* X, int r1, const double* Y, int r2, int n, double* Z) {
  if (ex.dry) return;
  const long total = (long)n * r1 * r2;
  const bool vec = (n % 2) == 0 && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y) |
                                     reinterpret_cast<uintptr_t>(Z)) & 15) == 0;
  if (vec) {
    const int h = n / 2;
    dim3 grid(std::max(1, std::min(ceil_div(h, 256), std::max(1, 4 * sm_count() / std::max(r1, 1)))), r1);
    TT_KERNEL(ex, K_OTHER, (double)total, 8.0 * ((double)n * (r1 + r2) + (double)total),
              k_khatri_rao2<<<grid, 256, 0, ex.s>>>(X, r1, Y, r2, n, Z));
    return;
  }
  TT_KERNEL(ex, K_OTHER, (double)total, 8.0 * ((double)n * (r1 + r2) + (double)total),
            k_khatri_rao<<<grid_for(total), 256, 0, ex.s>>>(X, r1, Y, r2, n, Z));
}

// ============================================================== sketch matrix
// Rademacher entries from SplitMix64 of (seed, index): a fixed deterministic
// test matrix for the randomized range finder.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ============================================================== transposes
template <typename Real>
__global__ void k_transpose(const Real* __restrict__ X, int m, int n, long ldx, Real* __restrict__ Y, long ldy) {
  __shared__ Real tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + dy;
    tile[dy][threadIdx.x] = (i < m && j < n) ? X[i + (size_t)j * ldx] : Real(0);
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int j = j0 + threadIdx.x, i = i0 + dy;
    if (i < m && j < n) Y[j + (size_t)i * ldy] = tile[threadIdx.x][dy];
  }
}
// Y (n x m) = X^T for X (m x n)
template <typename Real>
void transpose(Exec& ex, const Real* X, int m, int n, long ldx, Real* Y, long ldy) {
  if (ex.dry) return;
  dim3 grid(ceil_div(m, 32), ceil_div(n, 32));
  TT_KERNEL(ex, K_OTHER, 0, 2.0 * sizeof(Real) * m * (double)n,
            k_transpose<Real><<<grid, dim3(32, 8), 0, ex.s>>>(X, m, n, ldx, Y, ldy));
}
template void transpose<double>(Exec&, const double*, int, int, long, double*, long);
template void transpose<float>(Exec&, const float*, int, int, long, float*, long);

// ============================================================== sync helpers
int fetch_int(Exec& ex, const int* d) {
  if (ex.dry) return -1;
  TT_CUDA(cudaMemcpyAsync(ex.h_pinned, d, sizeof(int), cudaMemcpyDeviceToHost, ex.s));
  host_wait(ex);
  ex.syncs++;
  prof_flush(ex);
  return ex.h_pinned[0];
}
int fetch_svd_info(Exec& ex, const int* d, int p, const double* tail, double* tl) {
  if (ex.dry) {
    if (tl) tl[0] = tl[1] = 0.0;
    return -1;
  }
  TT_CUDA(cudaMemcpyAsync(ex.h_pinned, d, 3 * sizeof(int), cudaMemcpyDeviceToHost, ex.s));
  if (tail) TT_CUDA(cudaMemcpyAsync(ex.h_pinned_d, tail, 2 * sizeof(double), cudaMemcpyDeviceToHost, ex.s));
  host_wait(ex);
  if (tail) {
    tl[0] = ex.h_pinned_d[0];
    tl[1] = ex.h_pinned_d[1];
  }
  ex.syncs++;
  prof_flush(ex);
  ex.svd_calls++;
  ex.svd_p += p;
  ex.svd_pd += ex.h_pinned[1];
  ex.svd_sweeps += ex.h_pinned[2];
  ex.jacobi_sweeps += ex.h_pinned[2];
  return ex.h_pinned[0];
}

void fetch_doubles(Exec& ex, const double* d, int n, double* out) {
  if (ex.dry) {
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    return;
  }
  TT_REQUIRE(n <= 16, TT_ERR_ARG);
  TT_CUDA(cudaMemcpyAsync(ex.h_pinned_d, d, sizeof(double) * n, cudaMemcpyDeviceToHost, ex.s));
  host_wait(ex);
  ex.syncs++;
  prof_flush(ex);
  for (int i = 0; i < n; ++i) out[i] = ex.h_pinned_d[i];
}

// ============================================================== TT sums
// Up to kConcatMax terms of a sum concatenated in one launch: the first core
// of term t scaled by its coefficient into columns off_t.., the second core
// copied alike.
constexpr int kConcatMax = 8;
struct ConcatDesc {
  const double* a[kConcatMax];
  const double* b[kConcatMax];
  double c[kConcatMax];
  int off[kConcatMax + 1];  // column offsets; off[nt] = total rank
  int nt;
};

__global__ void k_concat(ConcatDesc d, int n1, int n2, double* __restrict__ A, double* __restrict__ B) {
  const long na = (long)n1 * d.off[d.nt], total = na + (long)n2 * d.off[d.nt];
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const bool first = t < na;
    const long u = first ? t : t - na;
    const int n = first ? n1 : n2;
    const int col = (int)(u / n), i = (int)(u - (long)col * n);
    int q = 0;
    while (q + 1 < d.nt && col >= d.off[q + 1]) ++q;
    const int lc = col - d.off[q];
    if (first)
      A[u] = d.c[q] * d.a[q][i + (size_t)lc * n1];
    else
      B[u] = d.b[q][i + (size_t)lc * n2];
  }
}

void tt_concat(Exec& ex, const std::vector<Term>& terms, TT& out) {
  int off = 0;
  for (const Term& t : terms) {
    TT_REQUIRE(t.x.n1 == out.n1 && t.x.n2 == out.n2, TT_ERR_ARG);
    TT_REQUIRE(off + t.x.r <= out.cap, TT_ERR_ARG);
    off += t.x.r;
  }
  out.r = off;
  if (ex.dry || off == 0) return;
  if ((int)terms.size() > kConcatMax) {
    int o = 0;
    for (const Term& t : terms) {
      scaled_copy(ex, out.a + (size_t)o * out.n1, t.x.a, (long)out.n1 * t.x.r, t.c);
      scaled_copy(ex, out.b + (size_t)o * out.n2, t.x.b, (long)out.n2 * t.x.r, 1.0);
      o += t.x.r;
    }
    return;
  }
  ConcatDesc d{};
  d.nt = 0;
  int o = 0;
  for (const Term& t : terms) {
    if (t.x.r == 0) continue;
    d.a[d.nt] = t.x.a;
    d.b[d.nt] = t.x.b;
    d.c[d.nt] = t.c;
    d.off[d.nt] = o;
    o += t.x.r;
    d.nt++;
  }
  d.off[d.nt] = o;
  const long total = (long)(out.n1 + out.n2) * o;
  TT_KERNEL(ex, K_OTHER, (double)out.n1 * o, 16.0 * total,
            k_concat<<<grid_for(total), 256, 0, ex.s>>>(d, out.n1, out.n2, out.a, out.b));
}

int total_rank(const std::vector<Term>& terms) {
  int r = 0;
  for (const Term& t : terms) r += t.x.r;
  return r;
}

// ============================================================== precision helpers
// The FP32 precision form runs the dense rounding contractions (formation,
// range-finder products, TSQR and its applications) on FP32 working copies;
// the small SVD and the output cores stay FP64.
template <typename D, typename S>
__global__ void k_convert(D* __restrict__ dst, const S* __restrict__ src, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    dst[t] = D(src[t]);
}
template <typename D, typename S>
static void convert(Exec& ex, D* dst, const S* src, long n) {
  if (n <= 0 || ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 0, (double)(sizeof(D) + sizeof(S)) * n,
            (k_convert<D, S><<<grid_for(n), 256, 0, ex.s>>>(dst, src, n)));
}
// X (n values, FP64) as a Real array: X itself for double, else a converted copy
template <typename Real>
static void copy_real(Exec& ex, Real* dst, const Real* src, long n) {
  if (ex.dry || n <= 0) return;
  TT_CUDA(cudaMemcpyAsync(dst, src, sizeof(Real) * n, cudaMemcpyDeviceToDevice, ex.s));
}
template <typename Real>
static const Real* as_real(Exec& ex, const double* X, long n) {
  if constexpr (std::is_same<Real, double>::value) {
    return X;
  } else {
    Real* y = ex.ar->get<Real>((size_t)n);
    convert(ex, y, X, n);
    return y;
  }
}
template <typename Real>
static const double* as_double(Exec& ex, const Real* X, long n) {
  if constexpr (std::is_same<Real, double>::value) {
    return X;
  } else {
    double* y = ex.ar->get<double>((size_t)n);
    convert(ex, y, X, n);
    return y;
  }
}
// Q [C; 0] into the FP64 core Out (m x k, ld m)
template <typename Real>
static void apply_to_core(Exec& ex, const QRTreeT<Real>& t, const double* C, int k, long ldc, double* Out) {
  tsqr_apply(ex, t, C, k, ldc, Out, (long)t.m);  // FP32 trees read C and write Out in FP64
}

// Working-precision product C = alpha A B + beta C of the rounding routes:
// FP64 and FP32 on CUDA cores; under TT_TF32 / TT_BF16 the larger FP32
// products go to the tensor cores (split operands, FP32-accurate).
template <typename Real>
static void lp_gemm(Exec& ex, int M, int N, int K, Real alpha, const Real* A, long ars, long acs, const Real* B,
                    long brs, long bcs, Real beta, Real* C, long ldc) {
  if constexpr (std::is_same<Real, float>::value) {
    if ((ex.precision == TT_TF32 || ex.precision == TT_BF16) && M >= 128 && K >= 32 &&
        (double)M * N * K >= 4.0e6) {
      tc_gemm<float>(ex, ex.precision, true, M, N, K, alpha, A, ars, acs, B, brs, bcs, beta, C, ldc);
      return;
    }
  }
  gemm<Real>(ex, M, N, K, alpha, A, ars, acs, B, brs, bcs, beta, C, ldc);
}

template <typename Real>
__global__ void k_rademacher(Real* __restrict__ O, long n, unsigned long long seed) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    O[t] = (splitmix64(seed * 0x100000000ull + (unsigned long long)t) >> 63) ? Real(1) : Real(-1);
}
template <typename Real>
__global__ void k_set_identity(Real* I, int p) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < p * p; t += gridDim.x * blockDim.x)
    I[t] = ((t % p) == (t / p)) ? Real(1) : Real(0);
}
template <typename Real>
static void set_identity_t(Exec& ex, Real* I, int p) {
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 0, (double)sizeof(Real) * p * p,
            k_set_identity<Real><<<grid_for((long)p * p), 256, 0, ex.s>>>(I, p));
}
void set_identity(Exec& ex, double* I, int p) { set_identity_t<double>(ex, I, p); }

// ============================================================== rounding
// residual target of the range finder: 1e-3 of the truncation tolerance, never
// looser than 1e-11 (so the result stays within 1e-10 of the exact truncated
// SVD) nor tighter than FP64 round-off of the residual itself
static double qb_target(double tol) { return std::max(std::min(1e-3 * tol, 1e-11), 4e-15); }
// FP32 working precision: the residual W0 - Q Q^T W0 formed in FP32 carries
// round-off of a few units of 2^-24 relative to ||W0||, so the range finder
// certifies at 4e-7, and truncation below 1e-6 would keep round-off directions
constexpr double kFp32QbFloor = 4e-7;
constexpr double kFp32TolFloor = 1e-6;
template <typename Real>
static double qb_target_t(double tol) {
  return std::is_same<Real, double>::value ? qb_target(tol) : std::max(qb_target(tol), kFp32QbFloor);
}
double effective_tol(const Exec& ex, double tol) {
  return ex.precision == TT_FP64 ? tol : std::max(tol, kFp32TolFloor);
}

static void finish_counts(Exec& ex, int k, int cap, int rin) {
  ex.rounds++;
  ex.last_rank = k;
  if (k == cap && rin > cap) ex.cap_hits++;
}

// First sketch of the range finder: cap + 8 columns (rounded to 8, at most
// 112 and the short mode s); the explicit residual check doubles it, up to
// 112, whenever the range is not yet captured (cap + 8 measured faster than
// 2 cap, cap and cap / 2 + 8 on the WENO5 workload: 129 vs 147 ms/step for
// cap, whose products retried 18 % more often).
static int rf_first_sketch(int s, int cap) { return std::min({112, s, ((cap + 8 + 7) / 8) * 8}); }

// Route of the rounding of a Hadamard product with R = r1 r2 terms.  The
// factored route (QR of both Khatri-Rao cores, SVD of an R x R factor) costs
// O(R^3) on one SM per factorisation; when both modes exceed 112 the
// alternative is the range finder on the formed product, whose cost is set by
// its sketch width p0 instead, and a product of smooth fields has far lower
// numerical rank than R, so the first sketch usually certifies.  On the 256^2
// faces (cap 32, p0 = 40) a factored rounding took 3.7 ms at R = 64 and
// 9-11 ms at R = 104-112, a range finder certified on its first sketch
// 3.6 ms, so the factored route is kept up to R = max(64, 1.5 p0).  (With
// 1.5 p0 alone, small rank caps sent products of R = 24-64 to sketches too
// narrow to certify: the 64-instance FP32 ensemble ran 1378 instead of
// 895 ms per step.)  (Sums keep the
// factored route up to R = 112: their terms are already rounded, so their
// numerical rank is close to R and the sketch would often have to grow.)
// Either route gives the truncated SVD, the range finder to within its
// certified residual.
static bool factored_route(int n1, int n2, int R, int cap) {
  const int s = std::min(n1, n2);
  if (R > 112 || R > s) return false;
  if (s <= 112) return true;  // the full route would be as exact and no cheaper
  return R <= 64 || 2 * R <= 3 * rf_first_sketch(s, cap);
}

// (i) Factored route, R <= 112 and R <= min(n1, n2): QR of both cores
// (TSQR), SVD of the R x R product of the triangular factors.
template <typename Real>
static RoundInfo round_factored(Exec& ex, const double* A, const double* B, int n1, int n2, int R, double tol,
                                int cap, TT& Y) {
  Scope sc(*ex.ar);
  // both cores factored side by side in shared launches (FP32 leaves
  // convert the FP64 cores on load)
  QRTreeT<Real> ta, tb;
  tsqr2(ex, A, n1, (long)n1, B, n2, (long)n2, R, ta, tb);
  Real* Mr = ex.ar->get<Real>((size_t)R * R);
  // M = R_A R_B^T
  gemm<Real>(ex, R, R, R, Real(1), ta.R, 1, R, tb.R, R, 1, Real(0), Mr, R);
  const double* M = as_double(ex, Mr, (long)R * R);
  debug_finite(ex, M, (long)R * R, "factored-route core M (n1, n2, R)", n1, n2, R);
  double* US = ex.ar->get<double>((size_t)R * R);
  double* V = ex.ar->get<double>((size_t)R * R);
  double* sig = ex.ar->get<double>(R);
  int* kd = ex.ar->get<int>(4);
  double* tail = ex.ar->get<double>(2);
  jacobi_svd(ex, M, R, tol, cap, US, V, sig, kd, tail);
  double tl[2];
  int k = fetch_svd_info(ex, kd, R, tail, tl);
  if (ex.dry) k = std::min(cap, R);
  tsqr_apply2(ex, ta, (const double*)US, (long)R, Y.a, (long)Y.n1, tb, (const double*)V, (long)R, Y.b,
              (long)Y.n2, k);
  Y.r = k;
  finish_counts(ex, k, cap, R);
  return RoundInfo{k, tl[0], tl[1], 0.0};
}

// (ii) Full-matrix routes on an explicit Y (n1 x n2): with s = min(n1, n2),
// the working matrix W0 is Y (s = n1) or Y^T (s = n2).
//   s <= 112: QR of W0^T (l x s) and SVD of R^T -- exact.
//   s  > 112: randomized range finder with an explicit residual check
//             ||W0 - Q Q^T W0||_F <= tau ||W0||_F, tau = qb_target(tol),
//             then QR of (Q^T W0)^T and SVD of the p x p factor (p <= 112).
template <typename Real>
static RoundInfo round_full_t(Exec& ex, const Real* Yf, int n1, int n2, double tol, int cap, TT& Y) {
  Scope sc(*ex.ar);
  const bool tr = n1 > n2;
  const int s = tr ? n2 : n1, l = tr ? n1 : n2;
  // W0(i, j), i < s, j < l
  const long wrs = tr ? n1 : 1, wcs = tr ? 1 : n1;
  double* Aw = tr ? Y.b : Y.a;  // s-side output core
  double* Bw = tr ? Y.a : Y.b;  // l-side output core
  double* kbuf = ex.ar->get<double>(4);
  int* kd = ex.ar->get<int>(4);
  double* tail = ex.ar->get<double>(2);
  if (s <= 112) {
    // W0^T (l x s) explicitly, col-major
    Real* WT = ex.ar->get<Real>((size_t)l * s);
    if (tr)
      convert(ex, WT, Yf, (long)l * s);  // Y itself is n1 x n2 = l x s
    else
      transpose(ex, Yf, n1, n2, n1, WT, l);
    QRTreeT<Real> tw;
    tsqr(ex, WT, l, s, l, tw);
    Real* Mr = ex.ar->get<Real>((size_t)s * s);
    transpose(ex, tw.R, s, s, s, Mr, s);  // M = R^T
    const double* M = as_double(ex, Mr, (long)s * s);
    debug_finite(ex, M, (long)s * s, "direct-route core M (n1, n2, s)", n1, n2, s);
    double* US = ex.ar->get<double>((size_t)s * s);
    double* V = ex.ar->get<double>((size_t)s * s);
    double* sig = ex.ar->get<double>(s);
    jacobi_svd(ex, M, s, tol, cap, US, V, sig, kd, tail);
    double tl[2];
    int k = fetch_svd_info(ex, kd, s, tail, tl);
    if (ex.dry) k = std::min(cap, s);
    // W0 = R^T Q_W^T = U S V^T Q_W^T: s-side core U S, l-side core Q_W V
    scaled_copy(ex, Aw, US, (long)s * k, 1.0);
    apply_to_core(ex, tw, V, k, s, Bw);
    Y.r = k;
    finish_counts(ex, k, cap, s);
    return RoundInfo{k, tl[0], tl[1], 0.0};
  }
  // ---- randomized range finder (s > 112)
  const double tau = qb_target_t<Real>(tol);
  sumsq(ex, Yf, n1, n2, n1, kbuf);  // ||W0||^2, read with the first residual
  double nrm2 = 0.0;
  int p = rf_first_sketch(s, cap);
  // a call site that keeps needing a wider sketch starts at the width that
  // certified its previous rounding
  if (ex.rf_hint && *ex.rf_hint > p) p = std::min({112, s, *ex.rf_hint});
  Real* Om = ex.ar->get<Real>((size_t)l * 112);
  Real* S = ex.ar->get<Real>((size_t)s * 112);
  Real* Q = ex.ar->get<Real>((size_t)s * 112);
  Real* WT = ex.ar->get<Real>((size_t)l * 112);
  Real* E = ex.ar->get<Real>((size_t)s * l);
  Real* I = ex.ar->get<Real>((size_t)112 * 112);
  double resid2 = 0.0;
  // SVD of Q^T W0 = WT^T = (Q_W R_W)^T = R_W^T Q_W^T for the current sketch
  QRTreeT<Real> tw;
  double* US = nullptr;
  double* V = nullptr;
  int k = 0;
  double tl[2] = {0.0, 0.0};
  auto svd_of_projection = [&] {
    tsqr(ex, WT, l, p, l, tw);
    Real* Mr = ex.ar->get<Real>((size_t)p * p);
    transpose(ex, tw.R, p, p, p, Mr, p);
    const double* M = as_double(ex, Mr, (long)p * p);
    debug_finite(ex, M, (long)p * p, "range-finder core M (n1, n2, p)", n1, n2, p);
    US = ex.ar->get<double>((size_t)p * p);
    V = ex.ar->get<double>((size_t)p * p);
    double* sig = ex.ar->get<double>(p);
    jacobi_svd(ex, M, p, tol, cap, US, V, sig, kd, tail);
    k = fetch_svd_info(ex, kd, p, tail, tl);
    if (ex.dry) k = std::min(cap, p);
  };
  for (int attempt = 0;; ++attempt) {
    ex.qb_attempts++;
    const size_t mk = ex.ar->mark();
    if (!ex.dry)
      TT_KERNEL(ex, K_OTHER, 0, (double)sizeof(Real) * l * p,
                k_rademacher<Real><<<grid_for((long)l * p), 256, 0, ex.s>>>(Om, (long)l * p, 0x7A3Dull + attempt));
    // S = W0 Om (s x p)
    lp_gemm<Real>(ex, s, p, l, Real(1), Yf, wrs, wcs, Om, 1, l, Real(0), S, s);
    QRTreeT<Real> ts;
    tsqr(ex, S, s, p, s, ts);
    // Q = Q_S [I_p; 0]
    set_identity_t(ex, I, p);
    tsqr_apply(ex, ts, I, p, p, Q, s);
    // WT = W0^T Q (l x p)
    lp_gemm<Real>(ex, l, p, s, Real(1), Yf, wcs, wrs, Q, 1, s, Real(0), WT, l);
    // E = W0 - Q WT^T
    if (tr)
      transpose(ex, Yf, n1, n2, n1, E, s);
    else
      convert(ex, E, Yf, (long)s * l);
    lp_gemm<Real>(ex, s, l, p, Real(-1), Q, 1, s, WT, l, 1, Real(1), E, s);
    sumsq(ex, E, s, l, s, kbuf + 1);
    double v[2];
    fetch_doubles(ex, kbuf, 2, v);
    nrm2 = v[0];
    resid2 = v[1];
    const bool ok = resid2 <= tau * tau * nrm2;
    const bool accept = ok || p >= std::min(112, s) || ex.dry;
    if (accept) {
      if (!ok && !ex.dry) ex.qb_uncertified++;
      if (ex.rf_hint && !ex.dry) *ex.rf_hint = p;
      // keep S/ts scratch alive: release nothing allocated after mark
      (void)mk;
      break;
    }
    ex.ar->reset(mk);
    // doubled (growing by half, 40 -> 64 -> 96, measured 10 % slower on the
    // WENO5 step: most lambda o jump products need more than 64 columns and
    // then took 96 instead of 80)
    p = std::min({112, s, 2 * p});
  }
  svd_of_projection();
  // s-side core Q (U S)_k, l-side core Q_W V_k
  if constexpr (std::is_same<Real, double>::value) {
    gemm(ex, s, k, p, 1.0, Q, 1, s, US, 1, p, 0.0, Aw, s);
  } else {
    const Real* USr = as_real<Real>(ex, US, (long)p * k);
    Real* Ar = ex.ar->get<Real>((size_t)s * k);
    lp_gemm<Real>(ex, s, k, p, Real(1), Q, 1, s, USr, 1, p, Real(0), Ar, s);
    convert(ex, Aw, Ar, (long)s * k);
  }
  apply_to_core(ex, tw, V, k, p, Bw);
  Y.r = k;
  finish_counts(ex, k, cap, s);
  return RoundInfo{k, std::sqrt(tl[0] * tl[0] + resid2), tl[1], std::sqrt(resid2)};
}

// (iii) Range finder on the cores (FP64), for an input Y = A B^T of R > 112
// columns whose modes both exceed 112 and whose n1 x n2 tensor would cost
// more to form and sketch than its cores: the steps of (ii) with every
// product taken through the cores, so Y is never formed.  With W0 = As Bl^T
// (As the s-side core, Bl the l-side core):
//   S  = As (Bl^T Om)                      the sketch,
//   C  = Q^T As,  WT = W0^T Q = Bl C^T      the projection,
//   ||W0||_F^2 = sum (As^T As) o (Bl^T Bl),
//   ||W0 - Q Q^T W0||_F^2 = sum (At^T At) o (Bl^T Bl),  At = As - Q C,
// the last two exact identities of the Frobenius norm of a product of
// cores.  At is formed in FP64 before its Gram, so the residual is resolved
// down to the round-off of At's entries (~1e-16 of ||As||), far below the
// certified 1e-11 relative residual; the sketch itself only has to span the
// range, which the residual check decides.
static double frf_flops(int s, int l, int R, int p) {
  return 2.0 * R * (double)R * (2.0 * s + l) + 2.0 * R * (double)p * (2.0 * l + 3.0 * s);
}
static double full_rf_flops(int n1, int n2, double form, int p) { return form + 6.0 * n1 * (double)n2 * p; }

// The same steps in the working precision Real: FP64, or FP32 for the
// precision forms, whose products (the cores' Grams, the sketch, the
// projections and At) go to the tcgen05 tensor cores under TT_TF32 / TT_BF16
// through lp_gemm (split operands, FP32-accurate); the p x p SVD stays FP64.
template <typename Real>
static RoundInfo round_factored_rf(Exec& ex, const double* A64, const double* B64, int n1, int n2, int R,
                                   double tol, int cap, TT& Y) {
  Scope sc(*ex.ar);
  const bool tr = n1 > n2;
  const int s = tr ? n2 : n1, l = tr ? n1 : n2;
  const Real* As = as_real<Real>(ex, tr ? B64 : A64, (long)s * R);
  const Real* Bl = as_real<Real>(ex, tr ? A64 : B64, (long)l * R);
  double* Aw = tr ? Y.b : Y.a;  // s-side output core
  double* Bw = tr ? Y.a : Y.b;  // l-side output core
  double* kbuf = ex.ar->get<double>(4);
  int* kd = ex.ar->get<int>(4);
  double* tail = ex.ar->get<double>(2);
  const double tau = qb_target_t<Real>(tol);
  // Grams of both cores and ||W0||^2
  Real* GB = ex.ar->get<Real>((size_t)R * R);
  Real* GA = ex.ar->get<Real>((size_t)R * R);
  lp_gemm<Real>(ex, R, R, l, Real(1), Bl, l, 1, Bl, 1, l, Real(0), GB, R);
  lp_gemm<Real>(ex, R, R, s, Real(1), As, s, 1, As, 1, s, Real(0), GA, R);
  const double* GB64 = as_double(ex, GB, (long)R * R);
  fdot(ex, as_double(ex, GA, (long)R * R), GB64, (long)R * R, kbuf);
  int p = rf_first_sketch(s, cap);
  if (ex.rf_hint && *ex.rf_hint > p) p = std::min({112, s, *ex.rf_hint});
  // the sizing pass takes the widest sketch the run may grow to (every
  // buffer, tree and product partial grows with p)
  if (ex.dry) p = std::min(112, s);
  Real* Om = ex.ar->get<Real>((size_t)l * 112);
  Real* T = ex.ar->get<Real>((size_t)R * 112);
  Real* S = ex.ar->get<Real>((size_t)s * 112);
  Real* Q = ex.ar->get<Real>((size_t)s * 112);
  Real* C = ex.ar->get<Real>((size_t)112 * R);
  Real* At = ex.ar->get<Real>((size_t)s * R);
  Real* GAt = ex.ar->get<Real>((size_t)R * R);
  Real* I = ex.ar->get<Real>((size_t)112 * 112);
  double nrm2 = 0.0, resid2 = 0.0;
  for (int attempt = 0;; ++attempt) {
    ex.qb_attempts++;
    const size_t mk = ex.ar->mark();
    if (!ex.dry)
      TT_KERNEL(ex, K_OTHER, 0, (double)sizeof(Real) * l * p,
                k_rademacher<Real><<<grid_for((long)l * p), 256, 0, ex.s>>>(Om, (long)l * p, 0x7A3Dull + attempt));
    // T = Bl^T Om (R x p), S = As T (s x p)
    lp_gemm<Real>(ex, R, p, l, Real(1), Bl, l, 1, Om, 1, l, Real(0), T, R);
    lp_gemm<Real>(ex, s, p, R, Real(1), As, 1, s, T, 1, R, Real(0), S, s);
    QRTreeT<Real> ts;
    tsqr(ex, S, s, p, s, ts);
    set_identity_t(ex, I, p);
    tsqr_apply(ex, ts, I, p, p, Q, s);
    // C = Q^T As (p x R); At = As - Q C; resid^2 = sum (At^T At) o GB
    lp_gemm<Real>(ex, p, R, s, Real(1), Q, s, 1, As, 1, s, Real(0), C, p);
    copy_real(ex, At, As, (long)s * R);
    lp_gemm<Real>(ex, s, R, p, Real(-1), Q, 1, s, C, 1, p, Real(1), At, s);
    lp_gemm<Real>(ex, R, R, s, Real(1), At, s, 1, At, 1, s, Real(0), GAt, R);
    fdot(ex, as_double(ex, GAt, (long)R * R), GB64, (long)R * R, kbuf + 1);
    double v[2];
    fetch_doubles(ex, kbuf, 2, v);
    nrm2 = v[0];
    resid2 = std::max(v[1], 0.0);
    const bool ok = resid2 <= tau * tau * nrm2;
    const bool accept = ok || p >= std::min(112, s) || ex.dry;
    if (accept) {
      if (!ok && !ex.dry) ex.qb_uncertified++;
      if (ex.rf_hint && !ex.dry) *ex.rf_hint = p;
      break;
    }
    ex.ar->reset(mk);
    p = std::min({112, s, 2 * p});
  }
  // WT = W0^T Q = Bl C^T (l x p); SVD of Q^T W0 = R_W^T Q_W^T (buffers
  // sized for the widest sketch: the sizing pass never widens it)
  Real* WT = ex.ar->get<Real>((size_t)l * 112);
  lp_gemm<Real>(ex, l, p, R, Real(1), Bl, 1, l, C, p, 1, Real(0), WT, l);
  QRTreeT<Real> tw;
  tsqr(ex, WT, l, p, l, tw);
  Real* Mr = ex.ar->get<Real>((size_t)112 * 112);
  transpose(ex, tw.R, p, p, p, Mr, p);
  const double* M = as_double(ex, Mr, (long)p * p);
  debug_finite(ex, M, (long)p * p, "factored range-finder core M (n1, n2, p)", n1, n2, p);
  double* US = ex.ar->get<double>((size_t)112 * 112);
  double* V = ex.ar->get<double>((size_t)112 * 112);
  double* sig = ex.ar->get<double>(112);
  jacobi_svd(ex, M, p, tol, cap, US, V, sig, kd, tail);
  double tl[2];
  int k = fetch_svd_info(ex, kd, p, tail, tl);
  if (ex.dry) k = std::min(cap, p);
  // s-side core Q (U S)_k, l-side core Q_W V_k
  if constexpr (std::is_same<Real, double>::value) {
    gemm(ex, s, k, p, 1.0, Q, 1, s, US, 1, p, 0.0, Aw, s);
  } else {
    const Real* USr = as_real<Real>(ex, US, (long)p * k);
    Real* Ar = ex.ar->get<Real>((size_t)s * std::max(k, 1));
    lp_gemm<Real>(ex, s, k, p, Real(1), Q, 1, s, USr, 1, p, Real(0), Ar, s);
    convert(ex, Aw, Ar, (long)s * k);
  }
  apply_to_core(ex, tw, V, k, p, Bw);
  Y.r = k;
  finish_counts(ex, k, cap, s);
  return RoundInfo{k, std::sqrt(tl[0] * tl[0] + resid2), tl[1], std::sqrt(resid2)};
}

RoundInfo round_full(Exec& ex, const double* Yf, int n1, int n2, double tol, int cap, TT& Y) {
  tol = effective_tol(ex, tol);
  if (ex.precision == TT_FP64) return round_full_t<double>(ex, Yf, n1, n2, tol, cap, Y);
  Scope sc(*ex.ar);
  return round_full_t<float>(ex, as_real<float>(ex, Yf, (long)n1 * n2), n1, n2, tol, cap, Y);
}

// Smallest column count R of an input whose rounding may take the range
// finder through the cores instead of the factored route (both modes above
// 112); TT_FRF_MIN_R (environment, read once) overrides it.
static int frf_min_r() {
  static const int v = [] {
    const char* e = std::getenv("TT_FRF_MIN_R");
    const int x = e ? std::atoi(e) : 0;
    return x >= 2 ? x : 113;
  }();
  return v;
}

template <typename Real>
static RoundInfo round_cores_t(Exec& ex, const double* A, const double* B, int n1, int n2, int R, double tol,
                               int cap, TT& Y) {
  {
    const int s = std::min(n1, n2), l = std::max(n1, n2), p = rf_first_sketch(s, cap);
    if (s > 112 && R >= frf_min_r() && frf_flops(s, l, R, p) < full_rf_flops(n1, n2, 2.0 * n1 * (double)n2 * R, p))
      return round_factored_rf<Real>(ex, A, B, n1, n2, R, tol, cap, Y);
  }
  if (R <= 112 && R <= std::min(n1, n2)) return round_factored<Real>(ex, A, B, n1, n2, R, tol, cap, Y);
  Scope sc(*ex.ar);
  Real* Yf = ex.ar->get<Real>((size_t)n1 * n2);
  if constexpr (std::is_same<Real, float>::value) {
    if (ex.precision == TT_TF32 || ex.precision == TT_BF16) {
      tc_gemm<double>(ex, ex.precision, true, n1, n2, R, 1.0f, A, 1, n1, B, n2, 1, 0.0f, Yf, n1);
      return round_full_t<Real>(ex, Yf, n1, n2, tol, cap, Y);
    }
  }
  const Real* Ar = as_real<Real>(ex, A, (long)n1 * R);
  const Real* Br = as_real<Real>(ex, B, (long)n2 * R);
  gemm<Real>(ex, n1, n2, R, Real(1), Ar, 1, n1, Br, n2, 1, Real(0), Yf, n1);
  return round_full_t<Real>(ex, Yf, n1, n2, tol, cap, Y);
}

RoundInfo round_cores(Exec& ex, const double* A, const double* B, int n1, int n2, int R, double tol, int cap,
                      TT& Y) {
  TT_REQUIRE(R >= 1 && cap >= 1 && Y.cap >= std::min(cap, std::max(1, std::min(n1, n2))), TT_ERR_ARG);
  debug_finite(ex, A, (long)n1 * R, "round_cores A (n1, n2, R)", n1, n2, R);
  debug_finite(ex, B, (long)n2 * R, "round_cores B (n1, n2, R)", n1, n2, R);
  tol = effective_tol(ex, tol);
  if (ex.precision == TT_FP64) return round_cores_t<double>(ex, A, B, n1, n2, R, tol, cap, Y);
  return round_cores_t<float>(ex, A, B, n1, n2, R, tol, cap, Y);
}

RoundInfo round_tt(Exec& ex, const TT& X, double tol, int cap, TT& Y) {
  return round_cores(ex, X.a, X.b, X.n1, X.n2, X.r, tol, cap, Y);
}

RoundInfo round_sum(Exec& ex, const std::vector<Term>& terms, double tol, int cap, TT& Y) {
  TT_REQUIRE(!terms.empty(), TT_ERR_ARG);
  Scope sc(*ex.ar);
  const int n1 = terms[0].x.n1, n2 = terms[0].x.n2;
  const int R = total_rank(terms);
  TT cat;
  cat.n1 = n1;
  cat.n2 = n2;
  cat.cap = R;
  cat.a = ex.ar->get<double>((size_t)n1 * R);
  cat.b = ex.ar->get<double>((size_t)n2 * R);
  tt_concat(ex, terms, cat);
  return round_tt(ex, cat, tol, cap, Y);
}

RoundInfo round_hadamard(Exec& ex, const TT& X, const TT& Z, double tol, int cap, TT& Y) {
  TT_REQUIRE(X.n1 == Z.n1 && X.n2 == Z.n2, TT_ERR_ARG);
  debug_finite(ex, X.a, (long)X.n1 * X.r, "round_hadamard X.a (n1, n2, r)", X.n1, X.n2, X.r);
  debug_finite(ex, X.b, (long)X.n2 * X.r, "round_hadamard X.b (n1, n2, r)", X.n1, X.n2, X.r);
  debug_finite(ex, Z.a, (long)Z.n1 * Z.r, "round_hadamard Z.a (n1, n2, r)", Z.n1, Z.n2, Z.r);
  debug_finite(ex, Z.b, (long)Z.n2 * Z.r, "round_hadamard Z.b (n1, n2, r)", Z.n1, Z.n2, Z.r);
  Scope sc(*ex.ar);
  const int n1 = X.n1, n2 = X.n2, R = X.r * Z.r;
  if (factored_route(n1, n2, R, cap)) {
    double* A = ex.ar->get<double>((size_t)n1 * R);
    double* B = ex.ar->get<double>((size_t)n2 * R);
    khatri_rao(ex, X.a, X.r, Z.a, Z.r, n1, A);
    khatri_rao(ex, X.b, X.r, Z.b, Z.r, n2, B);
    return round_cores(ex, A, B, n1, n2, R, tol, cap, Y);
  }
  tol = effective_tol(ex, tol);
  {
    // cores of the product (Khatri-Rao) and the range finder through them,
    // when that costs fewer flops than forming the n1 x n2 product
    const int s = std::min(n1, n2), l = std::max(n1, n2), p = rf_first_sketch(s, cap);
    if (s > 112 && frf_flops(s, l, R, p) < full_rf_flops(n1, n2, 2.0 * n1 * (double)n2 * (X.r + Z.r), p)) {
      double* A = ex.ar->get<double>((size_t)n1 * R);
      double* B = ex.ar->get<double>((size_t)n2 * R);
      khatri_rao(ex, X.a, X.r, Z.a, Z.r, n1, A);
      khatri_rao(ex, X.b, X.r, Z.b, Z.r, n2, B);
      if (ex.precision == TT_FP64) return round_factored_rf<double>(ex, A, B, n1, n2, R, tol, cap, Y);
      return round_factored_rf<float>(ex, A, B, n1, n2, R, tol, cap, Y);
    }
  }
  if (ex.precision == TT_FP64) {
    double* Yf = ex.ar->get<double>((size_t)n1 * n2);
    form_hadamard_full(ex, n1, n2, X.a, X.r, X.b, Z.a, Z.r, Z.b, Yf, n1);
    return round_full_t<double>(ex, Yf, n1, n2, tol, cap, Y);
  }
  float* Yf = ex.ar->get<float>((size_t)n1 * n2);
  form_hadamard_full(ex, n1, n2, X.a, X.r, X.b, Z.a, Z.r, Z.b, Yf, n1);
  return round_full_t<float>(ex, Yf, n1, n2, tol, cap, Y);
}

// ============================================================== misc
// sum_{i,j} X = (1^T A)(B^T 1) and ||X||_F^2 = sum (A^T A) o (B^T B): one CTA.
__global__ void k_tt_sum_norm(const double* __restrict__ A, const double* __restrict__ B, int n1, int n2, int r,
                              double* out) {
  __shared__ double ca[128], cb[128];
  __shared__ double red[33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = w; k < r; k += nw) {
    double sa = 0.0, sb = 0.0;
    for (int i = lane; i < n1; i += 32) sa += A[i + (size_t)k * n1];
    for (int j = lane; j < n2; j += 32) sb += B[j + (size_t)k * n2];
    for (int o = 16; o > 0; o >>= 1) {
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
      sb += __shfl_xor_sync(0xffffffffu, sb, o);
    }
    if (lane == 0) {
      ca[k] = sa;
      cb[k] = sb;
    }
  }
  __syncthreads();
  double s = 0.0;
  for (int k = threadIdx.x; k < r; k += blockDim.x) s = fma(ca[k], cb[k], s);
  // block reduce
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    out[0] = t;
  }
  __syncthreads();
  // Frobenius: sum_{k,l} (A^T A)_{kl} (B^T B)_{kl}
  double f = 0.0;
  for (int kl = w; kl < r * r; kl += nw) {
    const int k = kl % r, l2 = kl / r;
    double ga = 0.0, gb = 0.0;
    for (int i = lane; i < n1; i += 32) ga = fma(A[i + (size_t)k * n1], A[i + (size_t)l2 * n1], ga);
    for (int j = lane; j < n2; j += 32) gb = fma(B[j + (size_t)k * n2], B[j + (size_t)l2 * n2], gb);
    for (int o = 16; o > 0; o >>= 1) {
      ga += __shfl_xor_sync(0xffffffffu, ga, o);
      gb += __shfl_xor_sync(0xffffffffu, gb, o);
    }
    if (lane == 0) f = fma(ga, gb, f);
  }
  __syncthreads();
  if (lane == 0) red[w] = f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    out[1] = t > 0.0 ? sqrt(t) : 0.0;
  }
}

void tt_sum_norm(Exec& ex, const TT& X, double* out_dev) {
  TT_REQUIRE(X.r <= 128, TT_ERR_ARG);
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 2.0 * (X.n1 + X.n2) * (double)X.r * X.r, 8.0 * (X.n1 + X.n2) * (double)X.r,
            k_tt_sum_norm<<<1, 1024, 0, ex.s>>>(X.a, X.b, X.n1, X.n2, X.r, out_dev));
}

}  // namespace ttfv
