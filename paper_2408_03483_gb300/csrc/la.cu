// Dense FP64 building blocks of TT rounding and cross (Sec. 3.2-3.3):
// split-K GEMM, full Hadamard-product formation, sums of squares, Householder
// TSQR with implicit Q, one-sided Jacobi SVD, maximum-volume row selection.
//
// GB300 has 2 FP64 FMA/clk/SM (about 8 GFLOP/s per SM), so every kernel with
// real FP64 work spreads it over at least ~2 CTAs per SM (split-K, row
// blocks); the small dense factorisations (p <= 112) run one per CTA with the
// matrix resident in shared memory.
#include <cstdlib>
#include <cfloat>
#include <cmath>
#include <algorithm>
#include <type_traits>
#include <cooperative_groups.h>
#include <mutex>

#include "tt_common.cuh"

namespace ttfv {

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over aligned groups of H lanes (H a power of two <= 32); every lane of
// the warp must take part.
template <typename Real>
__device__ __forceinline__ Real group_sum(Real v, int H) {
  for (int o = H >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  `red` holds >= 33 doubles.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Smallest ||x|| for which a reflector is formed: below it ||x||^2 and the
// products that scale the reflector leave the normal range (FP64: 1e-290,
// FP32: 1e-34 for the squares), so the column is left as it is (tau = 0).
// The entries skipped are at least 1e-145 (FP64) / 1e-17 (FP32) in absolute
// size, far below the round-off of any block the rounding meets.
template <typename Real>
__host__ __device__ constexpr Real hh_safe_norm() {
  return sizeof(Real) == 8 ? Real(1e-145) : Real(1e-17);
}

// Householder reflector of x = [alpha; tail] with sigma = ||tail||^2 known in
// every lane: beta = -sign(alpha) ||x||, tau = (beta - alpha)/beta, scale =
// 1/(alpha - beta).  GB300 builds FP64 sqrt/division from its few FP64 FMA
// units, so lane 0 alone evaluates them and broadcasts the results.
template <typename Real>
__device__ __forceinline__ void householder_params(Real alpha, Real sigma, Real& beta, Real& tau,
                                                   Real& scale) {
  Real b = alpha, t = Real(0), sc = Real(0);
  if ((threadIdx.x & 31) == 0 && sigma > Real(0) && fma(alpha, alpha, sigma) >= hh_safe_norm<Real>() *
                                                                                 hh_safe_norm<Real>()) {
    const Real nrm = sqrt(fma(alpha, alpha, sigma));
    b = alpha >= Real(0) ? -nrm : nrm;
    const Real d = alpha - b;
    sc = Real(1) / d;
    t = -d / b;
  }
  beta = __shfl_sync(0xffffffffu, b, 0);
  tau = __shfl_sync(0xffffffffu, t, 0);
  scale = __shfl_sync(0xffffffffu, sc, 0);
}

// ============================================================== GEMM
// C = alpha * A B + beta * C with generic strides; tile 32x32, BK 16,
// 256 threads x 4 outputs; deterministic split-K through a partial buffer.
constexpr int GB = 32, GK = 16;

template <typename Real>
__global__ void __launch_bounds__(256) k_gemm_partial(int M, int N, int K, int kchunk,
                                                      const Real* __restrict__ A, long ars, long acs,
                                                      const Real* __restrict__ B, long brs, long bcs,
                                                      Real* __restrict__ P) {
  __shared__ Real As[GK][GB + 1];
  __shared__ Real Bs[GK][GB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * GB, j0 = blockIdx.y * GB;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  Real acc[2][2] = {{Real(0), Real(0)}, {Real(0), Real(0)}};
  for (int k0 = kb; k0 < ke; k0 += GK) {
    for (int t = threadIdx.x; t < GB * GK; t += 256) {
      int ii, kk;
      if (ars == 1) { ii = t % GB; kk = t / GB; } else { kk = t % GK; ii = t / GK; }
      const int gi = i0 + ii, gk = k0 + kk;
      As[kk][ii] = (gi < M && gk < ke) ? A[gi * ars + gk * acs] : Real(0);
    }
    for (int t = threadIdx.x; t < GB * GK; t += 256) {
      int jj, kk;
      if (brs == 1) { kk = t % GK; jj = t / GK; } else { jj = t % GB; kk = t / GB; }
      const int gj = j0 + jj, gk = k0 + kk;
      Bs[kk][jj] = (gj < N && gk < ke) ? B[gk * brs + gj * bcs] : Real(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const Real a0 = As[kk][tx], a1 = As[kk][tx + 16];
      const Real b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
  Real* Pz = P + (size_t)blockIdx.z * M * N;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + tx + 16 * u, j = j0 + ty + 16 * v;
      if (i < M && j < N) Pz[i + (size_t)j * M] = acc[u][v];
    }
}

template <typename Real>
__global__ void k_gemm_reduce(int M, int N, int nsplit, const Real* __restrict__ P, Real alpha, Real beta,
                              Real* __restrict__ C, long ldc) {
  const long total = (long)M * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    Real s = Real(0);
    for (int z = 0; z < nsplit; ++z) s += P[t + (size_t)z * total];
    const int i = int(t % M), j = int(t / M);
    Real* c = C + i + (size_t)j * ldc;
    *c = (beta == Real(0)) ? alpha * s : fma(alpha, s, beta * *c);
  }
}

template <typename Real>
void gemm(Exec& ex, int M, int N, int K, Real alpha, const Real* A, long ars, long acs, const Real* B, long brs, long bcs,
          Real beta, Real* C, long ldc) {
  if (M <= 0 || N <= 0) return;
  const int tiles = ceil_div(M, GB) * ceil_div(N, GB);
  // K split: the CTA count tiles * nsplit is balanced over the SMs (FP64
  // work per SM ~ the CTAs it holds, and one CTA already keeps an SM's FP64
  // pipes busy), so nsplit maximises tiles * nsplit / (SMs * ceil(tiles *
  // nsplit / SMs)) among the splits with K chunks of at least 64, at least
  // two CTAs per SM where K allows (latency of the tile loads), fewer
  // splits on ties
  const int sms = sm_count(), kmax = std::max(1, K / 64);
  int nsplit = 1;
  double best = -1.0;
  for (int ns = 1; ns <= std::min(kmax, 64); ++ns) {
    const long ctas = (long)tiles * ns;
    const double util = (double)ctas / ((double)sms * (double)((ctas + sms - 1) / sms));
    const double score = util * std::min(1.0, (double)ctas / (2.0 * sms));
    if (score > best + 1e-9) {
      best = score;
      nsplit = ns;
    }
  }
  int kchunk = ceil_div(ceil_div(std::max(K, 1), nsplit), GK) * GK;
  nsplit = ceil_div(std::max(K, 1), kchunk);
  Scope sc(*ex.ar);
  Real* P = ex.ar->get<Real>((size_t)nsplit * M * N);
  if (ex.dry) return;
  dim3 grid(ceil_div(M, GB), ceil_div(N, GB), nsplit);
  const double mnk = 2.0 * M * N * (double)K;
  TT_KERNEL(ex, K_GEMM, mnk, (double)sizeof(Real) * ((double)M * K + (double)K * N + (double)nsplit * M * N),
            k_gemm_partial<Real><<<grid, 256, 0, ex.s>>>(M, N, K, kchunk, A, ars, acs, B, brs, bcs, P));
  const long total = (long)M * N;
  const int blocks = std::max(1, std::min(ceil_div(total, 256), 4 * sm_count()));
  TT_KERNEL(ex, K_GEMM, (double)nsplit * total, (double)sizeof(Real) * total * (nsplit + (beta == Real(0) ? 1 : 2)),
            k_gemm_reduce<Real><<<blocks, 256, 0, ex.s>>>(M, N, nsplit, P, alpha, beta, C, ldc));
}

// ============================================================== Hadamard slab
// Y[i,j] = (A1 B1^T)[i,j] * (A2 B2^T)[i,j]: the full face tensor of a TT
// Hadamard product, formed without the r1*r2-column Khatri-Rao cores.
constexpr int HB = 32, HK = 16;
template <typename Real>
__global__ void __launch_bounds__(256) k_form_hadamard(int n1, int n2, const double* __restrict__ A1, int r1,
                                                       const double* __restrict__ B1,
                                                       const double* __restrict__ A2, int r2,
                                                       const double* __restrict__ B2, Real* __restrict__ Y,
                                                       long ldy) {
  __shared__ Real As[HK][HB + 1];
  __shared__ Real Bs[HK][HB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * HB, j0 = blockIdx.y * HB;
  Real acc[2][2][2] = {};
  for (int f = 0; f < 2; ++f) {
    const double* A = f ? A2 : A1;
    const double* B = f ? B2 : B1;
    const int r = f ? r2 : r1;
    for (int k0 = 0; k0 < r; k0 += HK) {
      for (int t = threadIdx.x; t < HB * HK; t += 256) {
        const int ii = t % HB, kk = t / HB;
        const int gi = i0 + ii, gj = j0 + ii, gk = k0 + kk;
        As[kk][ii] = (gi < n1 && gk < r) ? Real(A[gi + (size_t)gk * n1]) : Real(0);
        Bs[kk][ii] = (gj < n2 && gk < r) ? Real(B[gj + (size_t)gk * n2]) : Real(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < HK; ++kk) {
        const Real a0 = As[kk][tx], a1 = As[kk][tx + 16];
        const Real b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
        acc[f][0][0] = fma(a0, b0, acc[f][0][0]);
        acc[f][0][1] = fma(a0, b1, acc[f][0][1]);
        acc[f][1][0] = fma(a1, b0, acc[f][1][0]);
        acc[f][1][1] = fma(a1, b1, acc[f][1][1]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + tx + 16 * u, j = j0 + ty + 16 * v;
      if (i < n1 && j < n2) Y[i + (size_t)j * ldy] = acc[0][u][v] * acc[1][u][v];
    }
}

template <typename Real>
void form_hadamard_full(Exec& ex, int n1, int n2, const double* A1, int r1, const double* B1, const double* A2, int r2,
                        const double* B2, Real* Y, long ldy) {
  if (ex.dry) return;
  dim3 grid(ceil_div(n1, HB), ceil_div(n2, HB));
  TT_KERNEL(ex, K_FORM, 2.0 * n1 * (double)n2 * (r1 + r2) + (double)n1 * n2,
            8.0 * (double)(n1 + n2) * (r1 + r2) + (double)sizeof(Real) * n1 * n2,
            k_form_hadamard<Real><<<grid, 256, 0, ex.s>>>(n1, n2, A1, r1, B1, A2, r2, B2, Y, ldy));
}

// ============================================================== sum of squares
template <typename Real>
__global__ void k_sumsq_partial(const Real* __restrict__ X, int m, int n, long ld, double* part) {
  __shared__ double red[33];
  double s = 0.0;
  const long total = (long)m * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const double x = (double)X[(t % m) + (t / m) * ld];
    s = fma(x, x, s);
  }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_sum_fixed(const double* part, int n, double* out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int t = threadIdx.x; t < n; t += blockDim.x) s += part[t];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

template <typename Real>
void sumsq(Exec& ex, const Real* X, int m, int n, long ld, double* out) {
  Scope sc(*ex.ar);
  const int blocks = std::max(1, std::min(ceil_div((long)m * n, 256), 2 * sm_count()));
  double* part = ex.ar->get<double>(blocks);
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 2.0 * m * (double)n, (double)sizeof(Real) * m * (double)n,
            k_sumsq_partial<Real><<<blocks, 256, 0, ex.s>>>(X, m, n, ld, part));
  TT_KERNEL(ex, K_OTHER, blocks, 8.0 * blocks, k_sum_fixed<<<1, 256, 0, ex.s>>>(part, blocks, out));
}

// sum_t X[t] Y[t] over n contiguous entries, accumulated in FP64 with a fixed
// reduction order (two launches, like sumsq)
__global__ void k_fdot_partial(const double* __restrict__ X, const double* __restrict__ Y, long n, double* part) {
  __shared__ double red[33];
  double s = 0.0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    s = fma(X[t], Y[t], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

void fdot(Exec& ex, const double* X, const double* Y, long n, double* out) {
  Scope sc(*ex.ar);
  const int blocks = std::max(1, std::min(ceil_div(n, 256), 2 * sm_count()));
  double* part = ex.ar->get<double>(blocks);
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 2.0 * n, 16.0 * n, k_fdot_partial<<<blocks, 256, 0, ex.s>>>(X, Y, n, part));
  TT_KERNEL(ex, K_OTHER, blocks, 8.0 * blocks, k_sum_fixed<<<1, 256, 0, ex.s>>>(part, blocks, out));
}

// ============================================================== TSQR
// Tall-skinny QR: Householder QR of row blocks (leaves) held in shared
// memory, then trees of merges of their triangular factors; the reflectors
// are kept unnormalised (beta = -sign(alpha) ||x||, v = x - beta e_j,
// tau = 2 / v^T v = -1 / (beta (alpha - beta))).
constexpr int QR_THREADS = 512;
constexpr size_t QR_SMEM_MAX = 200 * 1024;

// lanes per column (K) and columns per warp (C) of the merge and apply-merge
// kernels for a triangle of order p, the merge's work warps and its padded
// shared-memory row length
struct MergeShape {
  int K, C, nwork, ld;
};
constexpr int AM_WARPS = 4;  // warps per CTA of the apply-merge kernel
__host__ __device__ inline int pow2_ceil(int x) {
  int v = 1;
  while (v < x) v <<= 1;
  return v;
}
inline MergeShape merge_shape(int p) {
  int C = pow2_ceil((p + 14) / 15);  // at most 15 work warps
  int K = 32 / C;
  if (K > pow2_ceil(p)) {
    K = pow2_ceil(p);
    C = 32 / K;
  }
  int ld = p;
  if (C < 16)
    while ((ld & 15) != C) ++ld;
  return MergeShape{K, C, (p + C - 1) / C, ld};
}

// Element i of an array that is FP64 (f64 != 0) or of the working type
template <typename Real>
__device__ __forceinline__ Real ld_any(const void* p, size_t i, int f64) {
  return f64 ? Real(static_cast<const double*>(p)[i]) : static_cast<const Real*>(p)[i];
}
template <typename Real>
__device__ __forceinline__ void st_any(void* p, size_t i, int f64, Real v) {
  if (f64)
    static_cast<double*>(p)[i] = double(v);
  else
    static_cast<Real*>(p)[i] = v;
}

// One matrix of a (one- or two-matrix) TSQR launch.  Launches carry two job
// descriptors; the CTAs of job 0 come first and a job with no CTAs (nb = 0,
// nodes = 0) is absent, so the two factorisations of a rounding share each
// launch and run side by side on the GPU.
template <typename Real>
struct LeafJob {
  const void* X;
  int x64;
  int m;
  long ldx;
  Real* V;
  Real* tau;
  Real* R;
  int nb;
};

// Householder QR of an mb x p row block (rows past m are zero) in shared
// memory, with the merge kernel's lane layout: the block row-major with the
// padded row length ld, lane (r, cc) of warp w owning column w C + cc and
// rows i = r (mod K), the reflector of column j formed by the scalar warp
// while the work warps form the dot products with the trailing columns.
// Reflectors are unnormalised, v = [alpha - beta at row j; A(j+1.., j)],
// tau = -1 / (beta (alpha - beta)); V keeps v below the diagonal and its top
// entry alpha - beta on the diagonal, R the upper triangle.
template <typename Real>
__global__ void __launch_bounds__(QR_THREADS) k_qr_blocks(LeafJob<Real> j0, LeafJob<Real> j1, int p, int mb, int K,
                                                          int ld) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Real* A = reinterpret_cast<Real*>(smraw);  // mb rows x ld
  __shared__ Real s_tau, s_vj, s_nrm;
  __shared__ Real s_vt[128];
  const bool second = (int)blockIdx.x >= j0.nb;
  const LeafJob<Real> jb = second ? j1 : j0;
  const int b = second ? (int)blockIdx.x - j0.nb : (int)blockIdx.x, r0 = b * mb;
  const int m = jb.m;
  for (int t = threadIdx.x; t < mb * p; t += blockDim.x) {
    const int i = t % mb, c = t / mb;
    A[(size_t)i * ld + c] = (r0 + i < m) ? ld_any<Real>(jb.X, (size_t)(r0 + i) + (size_t)c * jb.ldx, jb.x64) : Real(0);
  }
  const int C = 32 / K, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nwork = (int)(blockDim.x >> 5) - 1;
  const bool scalar = w == nwork;
  const int r = lane / C, c = w * C + lane % C;
  const int wlast = w * C + C - 1;
  __syncthreads();
  if (scalar && lane == 0) {
    Real sg = Real(0);
    for (int i = 1; i < mb; ++i) sg = fma(A[(size_t)i * ld], A[(size_t)i * ld], sg);
    s_nrm = sg;
  }
  __syncthreads();
  Real* tau_out = jb.tau + (size_t)b * p;
  for (int j = 0; j < p; ++j) {
    const bool busy = !scalar && wlast > j;  // warp-uniform
    const bool live = busy && c > j && c < p;
    const int i0 = j + 1 + ((r - j - 1) & (K - 1));  // first row > j of this lane's class
    Real d = Real(0);
    if (busy) {
      if (live)
        for (int i = i0; i < mb; i += K) d = fma(A[(size_t)i * ld + j], A[(size_t)i * ld + c], d);
      for (int o = C; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    } else if (scalar && lane == 0) {
      const Real sg = s_nrm;
      const Real alpha = A[(size_t)j * ld + j];
      Real tau = Real(0), vj = Real(0), beta = alpha;
      if (sg > Real(0) && fma(alpha, alpha, sg) >= hh_safe_norm<Real>() * hh_safe_norm<Real>()) {
        const Real nrm = sqrt(fma(alpha, alpha, sg));
        beta = alpha >= Real(0) ? -nrm : nrm;
        vj = alpha - beta;
        tau = Real(-1) / (beta * vj);
      }
      s_tau = tau;
      s_vj = vj;
      s_vt[j] = vj;
      tau_out[j] = tau;
      A[(size_t)j * ld + j] = beta;
    }
    __syncthreads();
    if (busy) {
      const Real tau = s_tau, vj = s_vj;
      const bool next = j + 1 < p && j + 1 >= w * C && j + 1 <= wlast;
      Real sq = Real(0);
      if (live) {
        Real* Aj = A + (size_t)j * ld + c;
        const Real f = tau * fma(vj, *Aj, d);
        if (next) {
          for (int i = i0; i < mb; i += K) {
            const Real x = fma(-f, A[(size_t)i * ld + j], A[(size_t)i * ld + c]);
            A[(size_t)i * ld + c] = x;
            if (i > j + 1) sq = fma(x, x, sq);
          }
        } else {
          for (int i = i0; i < mb; i += K) A[(size_t)i * ld + c] = fma(-f, A[(size_t)i * ld + j], A[(size_t)i * ld + c]);
        }
        if (r == 0) *Aj = fma(-f, vj, *Aj);
      }
      if (next) {
        for (int o = C; o < 32; o <<= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (c == j + 1 && r == 0) s_nrm = sq;
      }
    }
    __syncthreads();
  }
  Real* Vb = jb.V + (size_t)b * mb * p;
  for (int t = threadIdx.x; t < mb * p; t += blockDim.x) {
    const int i = t % mb, jj = t / mb;
    Vb[t] = (i > jj) ? A[(size_t)i * ld + jj] : (i == jj ? s_vt[jj] : Real(0));
  }
  Real* Rb = jb.R + (size_t)b * p * p;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int i = t % p, jj = t / p;
    Rb[t] = (i <= jj) ? A[(size_t)i * ld + jj] : Real(0);
  }
}

// Merge of up to g stacked upper-triangular factors [T; B_1; ...; B_{g-1}]
// (p x p each) by Householder reflectors that touch row j of T and rows 0..j
// of each B_b only.  Reflectors are kept unnormalised: v = [alpha - beta at T
// row j; B_b(0..j, j)], tau = -1 / (beta (alpha - beta)), so no scaling pass
// is needed.  A node with one input passes it through.
//
// Work layout (GB300 FP64: an SM sub-partition issues one FP64 warp
// instruction per ~64 cycles whatever the number of active lanes, so the
// kernel packs lanes and counts instructions):
// - the stacked blocks sit row-major in shared memory, row q = b p + i, with a
//   padded row length ld = p (mod 16 rule below), so lanes on consecutive
//   columns read consecutive words;
// - a lane owns column c = w C + (lane mod C) of its warp w and the row class
//   i = r (mod K), r = lane / C, of every bottom block (C K = 32), so one
//   column's K row classes live in one warp and its dot product is finished
//   by log2 K shuffle steps, with no shared-memory partials;
// - the last warp is the scalar warp: while the others form the dot products
//   of column j with the trailing columns, its lane 0 forms reflector j from
//   the norm that the owners of column j left at the end of the previous
//   column.  Two block barriers per column.
// ld = p rounded up to C (mod 16) when C < 16: lanes of a half warp then hold
// K/2 consecutive rows of C consecutive columns, i.e. 16 distinct banks.
template <typename Real>
struct MergeJob {
  const Real* Rin;
  int nin;
  int nodes;
  Real* Rout;
  Real* Vm;
  Real* vtop;
  Real* taum;
};

template <typename Real>
__global__ void __launch_bounds__(QR_THREADS) k_qr_merge(MergeJob<Real> j0, MergeJob<Real> j1, int p, int g, int K,
                                                         int ld) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Real* X = reinterpret_cast<Real*>(smraw);  // ng p rows x ld, row q = b p + i
  __shared__ Real s_tau, s_vj, s_nrm;
  const bool second = (int)blockIdx.x >= j0.nodes;
  const MergeJob<Real> jb = second ? j1 : j0;
  const int node = second ? (int)blockIdx.x - j0.nodes : (int)blockIdx.x;
  const int first = node * g, ng = min(g, jb.nin - first);
  Real* Ro = jb.Rout + (size_t)node * p * p;
  Real* Vo = jb.Vm + (size_t)node * g * p * p;  // bottom blocks 1..ng-1 at Vo + b p p
  Real* vt = jb.vtop + (size_t)node * p;
  Real* to = jb.taum + (size_t)node * p;
  const Real* __restrict__ Ri = jb.Rin + (size_t)first * p * p;
  if (ng == 1) {
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) Ro[t] = Ri[t];
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      to[j] = Real(0);
      vt[j] = Real(0);
    }
    return;
  }
  const int pp = p * p;
  for (int t = threadIdx.x; t < ng * pp; t += blockDim.x) {
    const int b = t / pp, rem = t - b * pp, i = rem % p, c = rem / p;
    X[(size_t)(b * p + i) * ld + c] = Ri[t];
  }
  const int C = 32 / K, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nwork = (int)(blockDim.x >> 5) - 1;
  const bool scalar = w == nwork;
  const int r = lane / C, c = w * C + lane % C;
  const int wlast = w * C + C - 1;  // the warp's last column
  __syncthreads();
  if (scalar && lane == 0) {
    Real sg = Real(0);
    for (int b = 1; b < ng; ++b) sg = fma(X[(size_t)b * p * ld], X[(size_t)b * p * ld], sg);
    s_nrm = sg;
  }
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    const bool busy = !scalar && wlast > j;  // warp-uniform
    const bool live = busy && c > j && c < p;
    Real d = Real(0);
    if (busy) {
      if (live)
        for (int b = 1; b < ng; ++b) {
          const Real* Xb = X + (size_t)b * p * ld;
          for (int i = r; i <= j; i += K) d = fma(Xb[(size_t)i * ld + j], Xb[(size_t)i * ld + c], d);
        }
      for (int o = C; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    } else if (scalar && lane == 0) {
      const Real sg = s_nrm;
      const Real alpha = X[(size_t)j * ld + j];
      Real tau = Real(0), vj = Real(0), beta = alpha;
      if (sg > Real(0) && fma(alpha, alpha, sg) >= hh_safe_norm<Real>() * hh_safe_norm<Real>()) {
        const Real nrm = sqrt(fma(alpha, alpha, sg));
        beta = alpha >= Real(0) ? -nrm : nrm;
        vj = alpha - beta;
        tau = Real(-1) / (beta * vj);
      }
      s_tau = tau;
      s_vj = vj;
      to[j] = tau;
      vt[j] = vj;
      X[(size_t)j * ld + j] = beta;
    }
    __syncthreads();
    if (busy) {
      const Real tau = s_tau, vj = s_vj;
      // the warp holding column j + 1 also sums the squares of what it
      // writes (warp-uniform; the other warps skip that FMA)
      const bool next = j + 1 < p && j + 1 >= w * C && j + 1 <= wlast;
      Real sq = Real(0);
      if (live) {
        Real* Tj = X + (size_t)j * ld + c;
        const Real f = tau * fma(vj, *Tj, d);
        for (int b = 1; b < ng; ++b) {
          Real* Xb = X + (size_t)b * p * ld;
          if (next) {
            for (int i = r; i <= j; i += K) {
              const Real x = fma(-f, Xb[(size_t)i * ld + j], Xb[(size_t)i * ld + c]);
              Xb[(size_t)i * ld + c] = x;
              sq = fma(x, x, sq);
            }
          } else {
            for (int i = r; i <= j; i += K)
              Xb[(size_t)i * ld + c] = fma(-f, Xb[(size_t)i * ld + j], Xb[(size_t)i * ld + c]);
          }
        }
        if (r == 0) *Tj = fma(-f, vj, *Tj);
      }
      // the owners of column j + 1 leave its norm below the diagonal (rows
      // 0..j just updated, row j + 1 untouched by reflector j) for the
      // scalar warp
      if (next) {
        for (int o = C; o < 32; o <<= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
        if (c == j + 1 && r == 0) {
          for (int b = 1; b < ng; ++b) {
            const Real x = X[(size_t)(b * p + j + 1) * ld + j + 1];
            sq = fma(x, x, sq);
          }
          s_nrm = sq;
        }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < pp; t += blockDim.x) {
    const int i = t % p, jj = t / p;
    Ro[t] = (i <= jj) ? X[(size_t)i * ld + jj] : Real(0);
  }
  for (int t = threadIdx.x; t < (ng - 1) * pp; t += blockDim.x) {
    const int b = 1 + t / pp, rem = t % pp, i = rem % p, jj = rem / p;
    Vo[(size_t)pp + t] = (i <= jj) ? X[(size_t)(b * p + i) * ld + jj] : Real(0);
  }
}

// fan-in of a merge node: as many triangles as the merge's and the
// apply-merge's shared memory hold, but at most 4 from p = 32 up and 16
// below: a lane's dot product runs over every bottom block of its column, so
// a level of small nodes on separate SMs beats one SM eliminating many
// triangles in turn
// TT_QR_FANIN (environment, read once): the largest merge fan-in from p = 32
// up (default 4), for tuning.
static int qr_fanin_cap() {
  static const int v = [] {
    const char* e = std::getenv("TT_QR_FANIN");
    const int x = e ? std::atoi(e) : 0;
    return x >= 2 ? x : 4;
  }();
  return v;
}
static int apply_merge_lanes(int p) { return std::min(32, pow2_ceil(p)); }
static int qr_merge_fanin(int p, size_t elem, int cap) {
  const MergeShape ms = merge_shape(p);
  const size_t per = (size_t)p * ms.ld * elem;
  const size_t per_apply = ((size_t)p * p + (size_t)AM_WARPS * p * (32 / apply_merge_lanes(p))) * elem;
  const int g = int(std::min(QR_SMEM_MAX / per, QR_SMEM_MAX / per_apply));
  return std::max(2, std::min(g, p >= 32 ? (cap >= 2 ? cap : qr_fanin_cap()) : 16));
}

// rows of a leaf: the leaf QR holds mb x ld entries, the leaf application mb x
// (p + 2 AM_WARPS) (its reflectors and four warps' two columns)
static int qr_leaf_rows(int p, size_t elem, int mult) {
  int mb = std::max(((p + 31) / 32) * 32, 64) * std::max(1, std::min(mult, 8));
  const size_t row = std::max<size_t>(merge_shape(p).ld, (size_t)p + 2 * AM_WARPS) * elem;
  const int lim = int((QR_SMEM_MAX - (size_t)p * elem) / row);
  return std::max(std::min(mb, lim), p);
}

// Factor nj (1 or 2) tall matrices with the same column count p: one leaf
// launch and one launch per merge level for both.
template <typename Real>
static void tsqr_run(Exec& ex, int nj, const void* const* X, const int* x64, const int* m, const long* ldx, int p,
                     QRTreeT<Real>* const* t) {
  TT_REQUIRE(p >= 1 && p <= 112, TT_ERR_ARG);
  const int mb = qr_leaf_rows(p, sizeof(Real), ex.qr_leaf_mult), g = qr_merge_fanin(p, sizeof(Real), ex.qr_fanin);
  Real* R[2] = {nullptr, nullptr};
  int n[2] = {1, 1};
  LeafJob<Real> lj[2] = {};
  int nbt = 0;
  double fl = 0.0, by = 0.0;
  for (int q = 0; q < nj; ++q) {
    TT_REQUIRE(m[q] >= 1, TT_ERR_ARG);
    QRTreeT<Real>& tq = *t[q];
    tq = QRTreeT<Real>{};
    tq.m = m[q];
    tq.p = p;
    tq.mb0 = mb;
    tq.nb0 = ceil_div(m[q], mb);
    tq.g = g;
    tq.V0 = ex.ar->get<Real>((size_t)tq.nb0 * mb * p);
    tq.tau0 = ex.ar->get<Real>((size_t)tq.nb0 * p);
    R[q] = ex.ar->get<Real>((size_t)tq.nb0 * p * p);
    lj[q] = LeafJob<Real>{X[q], x64[q], m[q], ldx[q], tq.V0, tq.tau0, R[q], tq.nb0};
    nbt += tq.nb0;
    n[q] = tq.nb0;
    fl += std::max(2.0 * m[q] * (double)p * p - tq.nb0 * (2.0 / 3.0) * p * (double)p * p, 0.0);
    by += (double)sizeof(Real) * ((double)m[q] * p * 2 + (double)tq.nb0 * p * p);
  }
  if (!ex.dry) {
    smem_attr_once(k_qr_blocks<Real>);
    const MergeShape ms = merge_shape(p);
    const size_t smem = (size_t)mb * ms.ld * sizeof(Real);
    TT_KERNEL(ex, K_QR, fl, by,
              k_qr_blocks<Real><<<nbt, 32 * (ms.nwork + 1), smem, ex.s>>>(lj[0], lj[1], p, mb, ms.K, ms.ld));
  }
  for (;;) {
    MergeJob<Real> mj[2] = {};
    int nodes_total = 0, maxin = 0;
    double mfl = 0.0, mby = 0.0;
    for (int q = 0; q < nj; ++q) {
      if (n[q] <= 1) continue;
      QRTreeT<Real>& tq = *t[q];
      const int nodes = (n[q] + g - 1) / g;
      Real* Vm = ex.ar->get<Real>((size_t)nodes * g * p * p);
      Real* vt = ex.ar->get<Real>((size_t)nodes * p);
      Real* tm = ex.ar->get<Real>((size_t)nodes * p);
      Real* Rn = ex.ar->get<Real>((size_t)nodes * p * p);
      tq.nin.push_back(n[q]);
      tq.Vm.push_back(Vm);
      tq.vtop.push_back(vt);
      tq.taum.push_back(tm);
      mj[q] = MergeJob<Real>{R[q], n[q], nodes, Rn, Vm, vt, tm};
      nodes_total += nodes;
      maxin = std::max(maxin, std::min(g, n[q]));
      mfl += (n[q] - nodes) * (2.0 / 3.0) * p * (double)p * p;
      mby += (double)sizeof(Real) * 3.0 * n[q] * p * (double)p;
      R[q] = Rn;
      n[q] = nodes;
    }
    if (nodes_total == 0) break;
    if (!ex.dry) {
      smem_attr_once(k_qr_merge<Real>);
      const MergeShape ms = merge_shape(p);
      const size_t smem = (size_t)maxin * p * ms.ld * sizeof(Real);
      TT_KERNEL(ex, K_QR_MERGE, mfl, mby,
                k_qr_merge<Real><<<nodes_total, 32 * (ms.nwork + 1), smem, ex.s>>>(mj[0], mj[1], p, g, ms.K, ms.ld));
    }
  }
  for (int q = 0; q < nj; ++q) t[q]->R = R[q];
}

template <typename Real, typename Src>
void tsqr(Exec& ex, const Src* X, int m, int p, long ldx, QRTreeT<Real>& t) {
  const void* xs[1] = {X};
  const int f64[1] = {std::is_same<Src, double>::value ? 1 : 0};
  const int ms[1] = {m};
  const long ls[1] = {ldx};
  QRTreeT<Real>* ts[1] = {&t};
  tsqr_run<Real>(ex, 1, xs, f64, ms, ls, p, ts);
}

template <typename Real, typename Src>
void tsqr2(Exec& ex, const Src* X1, int m1, long ldx1, const Src* X2, int m2, long ldx2, int p, QRTreeT<Real>& t1,
           QRTreeT<Real>& t2) {
  const void* xs[2] = {X1, X2};
  const int f = std::is_same<Src, double>::value ? 1 : 0;
  const int f64[2] = {f, f};
  const int ms[2] = {m1, m2};
  const long ls[2] = {ldx1, ldx2};
  QRTreeT<Real>* ts[2] = {&t1, &t2};
  tsqr_run<Real>(ex, 2, xs, f64, ms, ls, p, ts);
}

// Apply the level-0 reflectors of each block (in reverse order) to
// [Zin_block; 0], Zin_block = Zin + b*zstride (p x k, ld zld).  As in the
// apply-merge kernel, each warp takes C columns of Z through all p
// reflectors on its own (lane (r, cc) owning rows i = r (mod K) of column
// cc, K = 16), the leaf's reflectors staged in shared memory once per CTA,
// and a leaf's column groups spread over `cpn` CTAs.
template <typename Real>
struct ALeafJob {
  const Real* V;
  const Real* tau;
  int rows;
  int nb;
  const void* zin;
  int z64;
  long zstride, zld;
  void* out;
  int o64;
  long ldo;
};

constexpr int AL_LANES = 16;  // lanes per column of the leaf application

template <typename Real>
__global__ void __launch_bounds__(AM_WARPS * 32) k_qr_apply_blocks(ALeafJob<Real> j0, ALeafJob<Real> j1, int mb, int p,
                                                                  int k, int cpn) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int K = AL_LANES, C = 32 / AL_LANES;
  const int leafg = (int)blockIdx.x / cpn, part = (int)blockIdx.x - leafg * cpn;
  const bool second = leafg >= j0.nb;
  const ALeafJob<Real> jb = second ? j1 : j0;
  const int b = second ? leafg - j0.nb : leafg;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = lane / C, cc = lane % C;
  const int c = (part * AM_WARPS + w) * C + cc;  // this lane's column of Z
  const bool col = c < k;
  Real* V = reinterpret_cast<Real*>(smraw);  // mb x p, column-major, top entries on the diagonal
  Real* tv = V + (size_t)mb * p;
  {
    const Real* __restrict__ Vg = jb.V + (size_t)b * mb * p;
    for (int t = threadIdx.x; t < mb * p; t += blockDim.x) V[t] = Vg[t];
    for (int t = threadIdx.x; t < p; t += blockDim.x) tv[t] = jb.tau[(size_t)b * p + t];
  }
  __syncthreads();
  if ((part * AM_WARPS + w) * C >= k) return;  // warp-uniform: no column here
  Real* Z = tv + p + (size_t)w * mb * C;  // row i, C words per row
  const size_t zoff = (size_t)b * jb.zstride;
  for (int i = r; i < mb; i += K)
    Z[(size_t)i * C + cc] = (col && i < p) ? ld_any<Real>(jb.zin, zoff + i + (size_t)c * jb.zld, jb.z64) : Real(0);
  __syncwarp();
  for (int j = p - 1; j >= 0; --j) {
    const Real tj = tv[j];
    if (tj == Real(0)) continue;  // uniform across the warp
    const Real* v = V + (size_t)j * mb;
    const bool top = r == (j & (K - 1));  // owner of row j
    const int i0 = j + 1 + ((r - j - 1) & (K - 1));
    Real d = top ? v[j] * Z[(size_t)j * C + cc] : Real(0);
    for (int i = i0; i < mb; i += K) d = fma(v[i], Z[(size_t)i * C + cc], d);
    for (int o = C; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const Real f = tj * d;
    if (top) Z[(size_t)j * C + cc] = fma(-f, v[j], Z[(size_t)j * C + cc]);
    for (int i = i0; i < mb; i += K) Z[(size_t)i * C + cc] = fma(-f, v[i], Z[(size_t)i * C + cc]);
  }
  __syncwarp();
  if (col) {
    const int r0 = b * mb;
    for (int i = r; i < mb; i += K)
      if (r0 + i < jb.rows) st_any<Real>(jb.out, (size_t)(r0 + i) + (size_t)c * jb.ldo, jb.o64, Z[(size_t)i * C + cc]);
  }
}

// Reverse of a merge node: [top; B_1; ...] = Q_node [Z; 0; ...]; the top goes
// to input node*g, block b to input node*g + b (each p x k, ld p).
//
// The k columns of Z are independent under Q_node, so each warp takes C of
// them through all p reflectors on its own: lane (r, cc) = (lane / C,
// lane mod C) owns rows i = r (mod K) of every block of column cc (C K = 32,
// K the power of two >= p capped at 32), keeps them in its warp's slice of
// shared memory (row-major, C words per row, so a warp's 32 lanes touch 32
// consecutive words), and a dot product over the stacked rows is finished by
// log2 K shuffle steps.  The node's reflectors are copied to shared memory
// once per CTA; no block barrier inside the sweep.  A node's column
// groups are spread over `cpn` CTAs of up to four warps (one per SM
// sub-partition), so the p-reflector chains of a level's nodes run on many
// SMs at once.
template <typename Real>
struct AMergeJob {
  const Real* Vm;
  const Real* vtop;
  const Real* taum;
  int nin;
  int nodes;
  const void* zin;
  int z64;
  long zstride, zld;
  Real* zout;
};

template <typename Real>
__global__ void __launch_bounds__(AM_WARPS * 32) k_qr_apply_merge(AMergeJob<Real> j0, AMergeJob<Real> j1, int p,
                                                                  int g, int k, int K, int cpn) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nodeg = (int)blockIdx.x / cpn, part = (int)blockIdx.x - nodeg * cpn;
  const bool second = nodeg >= j0.nodes;
  const AMergeJob<Real> jb = second ? j1 : j0;
  const int node = second ? nodeg - j0.nodes : nodeg;
  const int first = node * g, ng = min(g, jb.nin - first);
  const size_t zoff = (size_t)node * jb.zstride;
  const long zld = jb.zld;
  Real* out = jb.zout + (size_t)first * p * k;
  const int C = 32 / K, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = lane / C, cc = lane % C;
  const int c = (part * AM_WARPS + w) * C + cc;  // this lane's column of Z
  const bool col = c < k;
  if (ng == 1) {
    if ((part * AM_WARPS + w) * C < k && col)
      for (int i = r; i < p; i += K) out[i + (size_t)c * p] = ld_any<Real>(jb.zin, zoff + i + (size_t)c * zld, jb.z64);
    return;
  }
  // the node's reflectors (bottom blocks 1..ng-1, column-major p x p) and
  // their top entries and factors, staged once for all of the CTA's warps
  const int nv = (ng - 1) * p * p;
  Real* V = reinterpret_cast<Real*>(smraw);
  Real* vt = V + nv;
  Real* tv = vt + p;
  {
    const Real* __restrict__ Vg = jb.Vm + (size_t)node * g * p * p + (size_t)p * p;
    for (int t = threadIdx.x; t < nv; t += blockDim.x) V[t] = Vg[t];
    for (int t = threadIdx.x; t < p; t += blockDim.x) {
      vt[t] = jb.vtop[(size_t)node * p + t];
      tv[t] = jb.taum[(size_t)node * p + t];
    }
  }
  __syncthreads();
  if ((part * AM_WARPS + w) * C >= k) return;  // warp-uniform: no column here
  Real* Z = tv + p + (size_t)w * ng * p * C;  // row q = b p + i, C words per row
  for (int q = r; q < ng * p; q += K)
    Z[(size_t)q * C + cc] = (col && q < p) ? ld_any<Real>(jb.zin, zoff + q + (size_t)c * zld, jb.z64) : Real(0);
  __syncwarp();
  for (int j = p - 1; j >= 0; --j) {
    const Real tj = tv[j];
    if (tj == Real(0)) continue;  // uniform across the warp
    const Real vj = vt[j];
    const bool top = r == (j & (K - 1));  // owner of top row j
    Real d = top ? vj * Z[(size_t)j * C + cc] : Real(0);
    for (int b = 1; b < ng; ++b) {
      const Real* Vb = V + (size_t)(b - 1) * p * p + (size_t)j * p;
      const Real* Zb = Z + (size_t)b * p * C + cc;
      for (int i = r; i <= j; i += K) d = fma(Vb[i], Zb[(size_t)i * C], d);
    }
    for (int o = C; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const Real f = tj * d;
    if (top) Z[(size_t)j * C + cc] = fma(-f, vj, Z[(size_t)j * C + cc]);
    for (int b = 1; b < ng; ++b) {
      const Real* Vb = V + (size_t)(b - 1) * p * p + (size_t)j * p;
      Real* Zb = Z + (size_t)b * p * C + cc;
      for (int i = r; i <= j; i += K) Zb[(size_t)i * C] = fma(-f, Vb[i], Zb[(size_t)i * C]);
    }
  }
  __syncwarp();
  if (col)
    for (int q = r; q < ng * p; q += K) {
      const int b = q / p, i = q - b * p;
      out[(size_t)b * p * k + i + (size_t)c * p] = Z[(size_t)q * C + cc];
    }
}

// Out_q (m_q x k) = Q_q [C_q; 0] for nj (1 or 2) trees with the same p:
// one launch per merge level (counted from the leaves) and one leaf launch.
template <typename Real>
static void tsqr_apply_run(Exec& ex, int nj, const QRTreeT<Real>* const* t, const void* const* C, const int* c64,
                           const long* ldc, void* const* Out, const int* o64, const long* ldo, int k) {
  const int p = t[0]->p;
  TT_REQUIRE(k >= 1 && k <= p && (nj == 1 || t[1]->p == p), TT_ERR_ARG);
  Scope sc(*ex.ar);
  const void* zin[2] = {C[0], nj > 1 ? C[1] : nullptr};
  int z64[2] = {c64[0], nj > 1 ? c64[1] : 0};
  long zs[2] = {0, 0}, zl[2] = {ldc[0], nj > 1 ? ldc[1] : 0};
  int L[2] = {0, 0}, maxL = 0;
  for (int q = 0; q < nj; ++q) {
    L[q] = (int)t[q]->nin.size();
    maxL = std::max(maxL, L[q]);
  }
  const int g = t[0]->g;
  for (int d = maxL - 1; d >= 0; --d) {
    AMergeJob<Real> aj[2] = {};
    int nodes_total = 0, maxin = 0;
    double fl = 0.0, by = 0.0;
    for (int q = 0; q < nj; ++q) {
      if (d >= L[q]) continue;
      const int nin = t[q]->nin[d], nodes = (nin + g - 1) / g;
      Real* zout = ex.ar->get<Real>((size_t)nin * p * k);
      aj[q] = AMergeJob<Real>{t[q]->Vm[d], t[q]->vtop[d], t[q]->taum[d], nin, nodes, zin[q], z64[q], zs[q], zl[q],
                              zout};
      nodes_total += nodes;
      maxin = std::max(maxin, std::min(g, nin));
      fl += (nin - nodes) * 2.0 * p * (double)p * k;
      by += (double)sizeof(Real) * ((double)nin * p * p + 2.0 * nin * p * k);
      zin[q] = zout;
      z64[q] = 0;
      zs[q] = (long)p * k;
      zl[q] = p;
    }
    if (!ex.dry && nodes_total > 0) {
      smem_attr_once(k_qr_apply_merge<Real>);
      const int K = apply_merge_lanes(p), C = 32 / K;
      const int cpn = ceil_div(ceil_div(k, C), AM_WARPS);
      const size_t smem = ((size_t)(maxin - 1) * p * p + 2 * (size_t)p + (size_t)AM_WARPS * maxin * p * C) * sizeof(Real);
      TT_KERNEL(ex, K_QR_APPLY_MERGE, fl, by,
                k_qr_apply_merge<Real><<<nodes_total * cpn, AM_WARPS * 32, smem, ex.s>>>(aj[0], aj[1], p, g, k, K,
                                                                                            cpn));
    }
  }
  ALeafJob<Real> lj[2] = {};
  int nbt = 0;
  double fl = 0.0, by = 0.0;
  for (int q = 0; q < nj; ++q) {
    const QRTreeT<Real>& tq = *t[q];
    lj[q] = ALeafJob<Real>{tq.V0, tq.tau0, tq.m, tq.nb0, zin[q], z64[q], zs[q], zl[q], Out[q], o64[q], ldo[q]};
    nbt += tq.nb0;
    fl += 4.0 * tq.m * (double)p * k;
    by += (double)sizeof(Real) * ((double)tq.m * (p + k) + (double)tq.nb0 * p * k);
  }
  if (!ex.dry) {
    const int mb = t[0]->mb0;
    smem_attr_once(k_qr_apply_blocks<Real>);
    const int cpn = ceil_div(ceil_div(k, 32 / AL_LANES), AM_WARPS);
    const size_t smem = ((size_t)mb * p + p + (size_t)AM_WARPS * mb * (32 / AL_LANES)) * sizeof(Real);
    TT_REQUIRE(smem <= QR_SMEM_MAX + 16 * 1024, TT_ERR_ARG);
    TT_KERNEL(ex, K_QR_APPLY, fl, by,
              k_qr_apply_blocks<Real><<<nbt * cpn, AM_WARPS * 32, smem, ex.s>>>(lj[0], lj[1], mb, p, k, cpn));
  }
}

template <typename Real, typename ZT, typename OT>
void tsqr_apply(Exec& ex, const QRTreeT<Real>& t, const ZT* C, int k, long ldc, OT* Out, long ldo) {
  const QRTreeT<Real>* ts[1] = {&t};
  const void* cs[1] = {C};
  const int c64[1] = {std::is_same<ZT, double>::value ? 1 : 0};
  const long lc[1] = {ldc};
  void* os[1] = {Out};
  const int o64[1] = {std::is_same<OT, double>::value ? 1 : 0};
  const long lo[1] = {ldo};
  tsqr_apply_run<Real>(ex, 1, ts, cs, c64, lc, os, o64, lo, k);
}

template <typename Real, typename ZT, typename OT>
void tsqr_apply2(Exec& ex, const QRTreeT<Real>& t1, const ZT* C1, long ldc1, OT* Out1, long ldo1,
                 const QRTreeT<Real>& t2, const ZT* C2, long ldc2, OT* Out2, long ldo2, int k) {
  const QRTreeT<Real>* ts[2] = {&t1, &t2};
  const void* cs[2] = {C1, C2};
  const int cf = std::is_same<ZT, double>::value ? 1 : 0, of = std::is_same<OT, double>::value ? 1 : 0;
  const int c64[2] = {cf, cf};
  const long lc[2] = {ldc1, ldc2};
  void* os[2] = {Out1, Out2};
  const int o64[2] = {of, of};
  const long lo[2] = {ldo1, ldo2};
  tsqr_apply_run<Real>(ex, 2, ts, cs, c64, lc, os, o64, lo, k);
}

// ---- explicit instantiations: FP64 path and the FP32 precision form
template void gemm<double>(Exec&, int, int, int, double, const double*, long, long, const double*, long, long, double,
                           double*, long);
template void gemm<float>(Exec&, int, int, int, float, const float*, long, long, const float*, long, long, float,
                          float*, long);
template void form_hadamard_full<double>(Exec&, int, int, const double*, int, const double*, const double*, int,
                                         const double*, double*, long);
template void form_hadamard_full<float>(Exec&, int, int, const double*, int, const double*, const double*, int,
                                        const double*, float*, long);
template void sumsq<double>(Exec&, const double*, int, int, long, double*);
template void sumsq<float>(Exec&, const float*, int, int, long, double*);
template void tsqr<double, double>(Exec&, const double*, int, int, long, QRTreeT<double>&);
template void tsqr<float, float>(Exec&, const float*, int, int, long, QRTreeT<float>&);
template void tsqr<float, double>(Exec&, const double*, int, int, long, QRTreeT<float>&);
template void tsqr2<double, double>(Exec&, const double*, int, long, const double*, int, long, int,
                                    QRTreeT<double>&, QRTreeT<double>&);
template void tsqr2<float, double>(Exec&, const double*, int, long, const double*, int, long, int, QRTreeT<float>&,
                                   QRTreeT<float>&);
template void tsqr_apply2<double, double, double>(Exec&, const QRTreeT<double>&, const double*, long, double*, long,
                                                  const QRTreeT<double>&, const double*, long, double*, long, int);
template void tsqr_apply2<float, double, double>(Exec&, const QRTreeT<float>&, const double*, long, double*, long,
                                                 const QRTreeT<float>&, const double*, long, double*, long, int);
template void tsqr_apply<double, double, double>(Exec&, const QRTreeT<double>&, const double*, int, long, double*,
                                                 long);
template void tsqr_apply<float, float, float>(Exec&, const QRTreeT<float>&, const float*, int, long, float*, long);
template void tsqr_apply<float, double, double>(Exec&, const QRTreeT<float>&, const double*, int, long, double*,
                                                long);

// ============================================================== small SVD
// SVD of a p x p matrix M (p <= 112) in one CTA, all in shared memory:
//  1. Householder QR with column pivoting of M^T, stopped once the trailing
//     Frobenius norm is <= defl ||M||_F (the deflated part joins the tail):
//     M = P L Q^T with L = R^T (p x pd) whose columns are graded;
//  2. one-sided (Hestenes) Jacobi on the pd columns of L, round-robin pairs,
//     one warp per pair; columns below defl ||M||_F are left untouched;
//  3. singular values = column norms, sorted; outputs P (L V) and Q V.
constexpr int SVD_THREADS = 1024;
constexpr int SVD_MAX_SWEEPS = 30;
constexpr int SVD_MIXED_MIN = 8;      // FP32 pre-rotation from this deflated rank up
constexpr int SVD_MIXED_SWEEPS = 6;   // cap of FP32 sweeps
constexpr float SVD_MIXED_TOL = 1e-5f;  // FP32 phase: rotate while |g| > 1e-5 sqrt(a b)
constexpr int SVD_CHOLQR_MIN = 60;      // deflated rank from which V0 is orthonormalised by Cholesky QR
constexpr int SVD_MAX_CLUSTER = 8;      // CTAs of the FP64 sweeps' cluster, at most
// FP64 scratch of one CTA: Householder vectors, taus, V0 (twice), G or T
__host__ __device__ inline size_t svd_scratch_doubles(int p) { return (size_t)4 * p * p + p; }

__global__ void __launch_bounds__(SVD_THREADS) k_svd_small(const double* __restrict__ Min, int p, double tol, int cap,
                                                          double defl, double* US, double* Vout, double* sig,
                                                          int* info, double* tail_out, double* scr,
                                                          unsigned* status) {
  extern __shared__ double sm[];
  double* A = sm;                  // p x p
  double* J = sm + (size_t)p * p;  // p x p scratch, then pd x pd Jacobi V
  __shared__ double cn[128];
  __shared__ double cn0[128];  // norms at the last exact computation
  __shared__ int piv[128];
  __shared__ int order[128];
  __shared__ double s_tau, s_fro2, s_trail;
  __shared__ int s_jmax, s_stop, s_rot, s_k, s_tmax, s_bad;
  __shared__ float cnf[128];
  __shared__ double gam[64], rc_c[64], rc_s[64];  // per pair of a round (q/2 <= 56)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // a launch over a cluster of cl CTAs: every CTA runs the same steps on the
  // same data up to the FP64 sweeps, each in its own slice of the scratch
  // (the grid is one cluster: rank = blockIdx.x; cluster calls only when cl > 1)
  namespace cg = cooperative_groups;
  const int cl = (int)gridDim.x, me = (int)blockIdx.x;
  scr += (size_t)me * svd_scratch_doubles(p);
  double* HV = scr;                  // Householder vectors, p x p
  double* htau = scr + (size_t)p * p;
  double* Vg = htau + p;             // pre-rotation scratch: pd x pd
  double* Gg = Vg + (size_t)p * p;   // pd x pd
  double* Tg = Gg + (size_t)p * p;   // p x pd

  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int i = t % p, j = t / p;
    A[t] = Min[j + (size_t)i * p];  // A = M^T
  }
  for (int j = threadIdx.x; j < p; j += blockDim.x) piv[j] = j;
  __syncthreads();
  for (int j = w; j < p; j += nw) {
    double s = 0.0;
    for (int i = lane; i < p; i += 32) s = fma(A[i + (size_t)j * p], A[i + (size_t)j * p], s);
    s = warp_sum(s);
    if (lane == 0) {
      cn[j] = s;
      cn0[j] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double f = 0.0;
    for (int j = 0; j < p; ++j) f += cn[j];
    s_fro2 = f;
  }
  __syncthreads();
  const double fro2 = s_fro2;
  if (!isfinite(fro2)) {
    // NaN/Inf input: flag it and return a rank-1 zero factorisation instead
    // of letting non-finite norms drive the pivot and sort indices (CTA 0;
    // the others leave: no cluster barrier has been reached)
    if (me != 0) return;
    for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
      US[t] = 0.0;
      Vout[t] = ((t % p) == (t / p)) ? 1.0 : 0.0;
    }
    for (int c = threadIdx.x; c < p; c += blockDim.x) sig[c] = 0.0;
    if (threadIdx.x == 0) {
      info[0] = 1;
      info[1] = 0;
      info[2] = 0;
      tail_out[0] = 0.0;
      tail_out[1] = 0.0;
      atomicOr(status, DEV_NONFINITE);
    }
    return;
  }
  const double thr = defl * defl * fro2;
  // ---- 1. QR with column pivoting of M^T, deflated.  The pivot search
  // runs on FP32 copies of the squared column norms scaled by 1/||M||_F^2
  // (it only picks a column); the stop test sums the FP64 norms whenever the
  // FP32 sum of the trailing norms is within a factor of 4 of the threshold.
  // The trailing columns are updated by warps that each own Cp columns and,
  // per column, the rows i = rp (mod Kp) below the pivot row, inner products
  // finished by shuffles.
  const double ifro2 = fro2 > 0.0 ? 1.0 / fro2 : 0.0;
  for (int j = threadIdx.x; j < p; j += blockDim.x) cnf[j] = (float)(cn[j] * ifro2);
  __syncthreads();
  const float thrf = (float)(thr * ifro2);
  // lane (rp, cp) = (lane mod Kp, lane / Kp): a half warp holds two columns'
  // eight consecutive row classes, so it touches at most two banks' worth of
  // columns whatever p
  constexpr int Kp = 8, Cp = 32 / Kp;
  const int rp = lane % Kp, cp = lane / Kp;
  int pd = p;
  for (int k = 0; k < p; ++k) {
    if (w == 0) {
      float best = -1.0f, tf = 0.0f;
      int bj = k;
      for (int j = k + lane; j < p; j += 32) {
        tf += cnf[j];
        if (cnf[j] > best) {
          best = cnf[j];
          bj = j;
        }
      }
      tf = warp_sum(tf);
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && oj < bj)) {
          best = ob;
          bj = oj;
        }
      }
      int stop = 0;
      double trail = 0.0;
      if (!(tf > 4.0f * thrf)) {  // near the threshold: decide in FP64
        for (int j = k + lane; j < p; j += 32) trail += cn[j];
        trail = warp_sum(trail);
        stop = trail <= thr ? 1 : 0;
      }
      if (lane == 0) {
        s_jmax = bj;
        s_stop = stop;
        s_trail = trail;
      }
    }
    __syncthreads();
    if (s_stop) {
      pd = k;
      break;
    }
    const int jm = s_jmax;
    if (jm != k) {
      for (int i = threadIdx.x; i < p; i += blockDim.x) {
        const double x = A[i + (size_t)k * p];
        A[i + (size_t)k * p] = A[i + (size_t)jm * p];
        A[i + (size_t)jm * p] = x;
      }
      if (threadIdx.x == 0) {
        const int t = piv[k];
        piv[k] = piv[jm];
        piv[jm] = t;
        const double c = cn[k];
        cn[k] = cn[jm];
        cn[jm] = c;
        const double c0 = cn0[k];
        cn0[k] = cn0[jm];
        cn0[jm] = c0;
        const float cf = cnf[k];
        cnf[k] = cnf[jm];
        cnf[jm] = cf;
      }
    }
    __syncthreads();
    double* col = A + (size_t)k * p;
    if (w == 0) {
      double sg = 0.0;
      for (int i = k + 1 + lane; i < p; i += 32) sg = fma(col[i], col[i], sg);
      sg = warp_sum(sg);
      const double alpha = col[k];
      double tau, beta, scale;
      householder_params(alpha, sg, beta, tau, scale);
      if (sg > 0.0)
        for (int i = k + 1 + lane; i < p; i += 32) col[i] *= scale;
      if (lane == 0) {
        col[k] = beta;
        s_tau = tau;
        htau[k] = tau;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    const int nact = p - k - 1;
    const int i0 = k + 1 + ((rp - k - 1) & (Kp - 1));  // first row > k of this lane's class
    for (int base = w * Cp; base < nact; base += nw * Cp) {  // warp-uniform
      const int c = k + 1 + base + cp;
      const bool colv = base + cp < nact;
      double* ccol = A + (size_t)(colv ? c : k) * p;
      if (tau != 0.0) {
        double d = 0.0;
        if (colv)
          for (int i = i0; i < p; i += Kp) d = fma(col[i], ccol[i], d);
        for (int o = 1; o < Kp; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        const double f = colv ? tau * (d + ccol[k]) : 0.0;
        __syncwarp();  // the column's lanes have read ccol[k]
        if (colv) {
          if (rp == 0) ccol[k] -= f;
          for (int i = i0; i < p; i += Kp) ccol[i] = fma(-f, col[i], ccol[i]);
        }
        __syncwarp();
      }
      // trailing norm below row k: downdate by the new row-k entry (one lane
      // per column), recompute exactly only after heavy cancellation (as
      // pivoted Householder QR codes do)
      double s2 = 0.0;
      int redo = 0;
      if (colv && rp == 0) {
        s2 = fma(-ccol[k], ccol[k], cn[c]);
        redo = (s2 <= 1e-6 * cn0[c]) ? 1 : 0;
      }
      redo = __shfl_sync(0xffffffffu, redo, cp * Kp);
      if (__any_sync(0xffffffffu, redo)) {
        double e = 0.0;
        if (colv && redo)
          for (int i = i0; i < p; i += Kp) e = fma(ccol[i], ccol[i], e);
        for (int o = 1; o < Kp; o <<= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if (colv && redo && rp == 0) {
          s2 = e;
          cn0[c] = e;
        }
      }
      if (colv && rp == 0) {
        cn[c] = s2 > 0.0 ? s2 : 0.0;
        cnf[c] = (float)(cn[c] * ifro2);
      }
    }
    __syncthreads();
  }
  const double qr_tail2 = (pd < p) ? s_trail : 0.0;
  // save the reflectors (below-diagonal parts) for the right factor
  for (int t = threadIdx.x; t < p * pd; t += blockDim.x) {
    const int i = t % p, kk = t / p;
    HV[t] = (i > kk) ? A[t] : 0.0;
  }
  // ---- 2. L = R^T (p x pd) into J, then back into A
  for (int t = threadIdx.x; t < p * pd; t += blockDim.x) {
    const int jr = t % p, i = t / p;
    J[t] = (i <= jr) ? A[i + (size_t)jr * p] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * pd; t += blockDim.x) A[t] = J[t];
  __syncthreads();
  for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) J[t] = ((t % pd) == (t / pd)) ? 1.0 : 0.0;
  __syncthreads();
  const int q = pd + (pd & 1);
  // a round's q/2 pairs take one warp each up to one pair per warp, and half
  // a warp each beyond (p > 64), so that a round is one pass of the warps
  const int H = (q / 2 > nw) ? 16 : 32, PW = 32 / H;
  const int sub = lane & (H - 1), lead = lane & ~(H - 1);
  // ---- 2a. FP32 pre-rotation.  One-sided Jacobi sweeps on an FP32 copy of L
  // (FP32 instructions cost 1/64 of FP64 ones here) orthogonalise its columns
  // to FP32 level; the accumulated rotations V0 are re-orthonormalised in FP64
  // (two Newton-Schulz steps V <- V (3 I - V^T V) / 2) and L <- L V0.  The
  // FP64 sweeps below then start from near-orthogonal columns, where they
  // converge in one or two sweeps; their result is the FP64 SVD whatever V0.
  if (pd >= SVD_MIXED_MIN) {
    float* Af = reinterpret_cast<float*>(J);  // p x pd floats, then pd x pd
    float* Jf = Af + (size_t)p * pd;          // fits: J holds p*p doubles
    // a power-of-two scale keeps the FP32 copy in range (rotations do not
    // depend on the scale)
    const double fscale = ldexp(1.0, -ilogb(sqrt(fro2)));
    for (int t = threadIdx.x; t < p * pd; t += blockDim.x) Af[t] = (float)(A[t] * fscale);
    for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) Jf[t] = ((t % pd) == (t / pd)) ? 1.0f : 0.0f;
    __syncthreads();
    const float epsf = SVD_MIXED_TOL;
    for (int sw = 0; sw < SVD_MIXED_SWEEPS; ++sw) {
      for (int j = w; j < pd; j += nw) {
        float sq = 0.0f;
        for (int r = lane; r < p; r += 32) sq = fmaf(Af[r + (size_t)j * p], Af[r + (size_t)j * p], sq);
        sq = warp_sum(sq);
        if (lane == 0) cnf[j] = sq;
      }
      if (threadIdx.x == 0) s_rot = 0;
      __syncthreads();
      for (int step = 0; step < q - 1; ++step) {
        // PW pairs per warp, H lanes each (the loop is warp-uniform: the
        // halves of a warp finish their sums by shuffles together)
        for (int base = w * PW; base < q / 2; base += nw * PW) {
          const int pr = base + lane / H;
          int i = 0, j = 0;
          bool ok = pr < q / 2;
          if (ok) {
            i = (pr == 0) ? 0 : 1 + ((pr - 1 + step) % (q - 1));
            j = 1 + ((q - 1 - pr - 1 + step) % (q - 1));
            ok = i < pd && j < pd;
          }
          float* ci = Af + (size_t)(ok ? i : 0) * p;
          float* cj = Af + (size_t)(ok ? j : 0) * p;
          float ga = 0.0f;
          if (ok)
            for (int r = sub; r < p; r += H) ga = fmaf(ci[r], cj[r], ga);
          ga = group_sum(ga, H);
          const float al = ok ? cnf[i] : 0.0f, be = ok ? cnf[j] : 0.0f;
          const bool rot = ok && (ga * ga > epsf * epsf * al * be);
          float c = 1.0f, sn = 0.0f;
          if (rot && sub == 0) {
            const float dd = be - al;
            const float t = (dd >= 0.0f ? 2.0f * ga : -2.0f * ga) / (fabsf(dd) + sqrtf(fmaf(dd, dd, 4.0f * ga * ga)));
            c = rsqrtf(fmaf(t, t, 1.0f));
            sn = c * t;
            cnf[i] = fmaf(-t, ga, al);
            cnf[j] = fmaf(t, ga, be);
          }
          c = __shfl_sync(0xffffffffu, c, lead);
          sn = __shfl_sync(0xffffffffu, sn, lead);
          if (rot) {
            for (int r = sub; r < p; r += H) {
              const float x = ci[r], y = cj[r];
              ci[r] = c * x - sn * y;
              cj[r] = sn * x + c * y;
            }
            float* vi = Jf + (size_t)i * pd;
            float* vj = Jf + (size_t)j * pd;
            for (int r = sub; r < pd; r += H) {
              const float x = vi[r], y = vj[r];
              vi[r] = c * x - sn * y;
              vj[r] = sn * x + c * y;
            }
            if (sub == 0) s_rot = 1;
          }
        }
        __syncthreads();
      }
      if (s_rot == 0) break;
      __syncthreads();
    }
    // V0 made orthonormal in FP64: by two Newton-Schulz steps
    // V <- V (3 I - V^T V) / 2 up to pd = SVD_CHOLQR_MIN, above by a Cholesky QR
    // (a quarter of the FP64 work, but 2 pd block barriers and a sequential
    // substitution, which only pay off for large pd)
    if (pd < SVD_CHOLQR_MIN) {
      for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) Vg[t] = (double)Jf[t];
      __syncthreads();
      for (int it = 0; it < 2; ++it) {
        const double* Vs = (it == 0) ? Vg : J;
        double* Vd = (it == 0) ? J : Vg;
        for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) {  // G = V^T V
          const int a = t % pd, b = t / pd;
          double g = 0.0;
          for (int r = 0; r < pd; ++r) g = fma(Vs[r + (size_t)a * pd], Vs[r + (size_t)b * pd], g);
          Gg[t] = g;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) {  // Vd = 1.5 V - 0.5 V G
          const int r = t % pd, b = t / pd;
          double u = 0.0;
          for (int a = 0; a < pd; ++a) u = fma(Vs[r + (size_t)a * pd], Gg[a + (size_t)b * pd], u);
          Vd[t] = fma(-0.5, u, 1.5 * Vs[t]);
        }
        __syncthreads();
      }
      for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) J[t] = Vg[t];
      __syncthreads();
    } else {
      // V0 in FP64, made orthonormal by a Cholesky QR: V0 is orthogonal to
      // FP32 round-off, so G = V0^T V0 = I + O(1e-7) is perfectly conditioned
      // and Q = V0 C^-T (G = C C^T, C lower) is orthonormal to FP64 round-off,
      // for a quarter of the FP64 work of two Newton-Schulz steps.  V0 goes to
      // global scratch twice: row-major in Vg (lanes along a row form G) and
      // column-major in Tg (lanes along a column solve for Q in place).
      for (int t = threadIdx.x; t < pd * pd; t += blockDim.x) {
        const int r = t % pd, a = t / pd;
        const double v = (double)Jf[t];
        Vg[a + (size_t)r * pd] = v;
        Tg[t] = v;
      }
      if (threadIdx.x == 0) s_bad = 0;
      __syncthreads();
      // lower triangle of G into J: a warp per column b, lanes over rows a >= b
      for (int b = w; b < pd; b += nw)
        for (int a = b + lane; a < pd; a += 32) {
          double g0 = 0.0, g1 = 0.0;
          int r = 0;
          for (; r + 1 < pd; r += 2) {
            g0 = fma(Vg[a + (size_t)r * pd], Vg[b + (size_t)r * pd], g0);
            g1 = fma(Vg[a + (size_t)(r + 1) * pd], Vg[b + (size_t)(r + 1) * pd], g1);
          }
          if (r < pd) g0 = fma(Vg[a + (size_t)r * pd], Vg[b + (size_t)r * pd], g0);
          J[a + (size_t)b * pd] = g0 + g1;
        }
      __syncthreads();
      // right-looking Cholesky over G's lower triangle: column k of C is
      // column k of G over sqrt(G[k][k]); 1 / C[k][k] is kept in cn0[k] (J's
      // diagonal is not read again)
      for (int k = 0; k < pd; ++k) {
        const double gkk = J[k + (size_t)k * pd];
        const bool okk = gkk > 0.5;  // a diagonal far from 1: V0 is not near-orthogonal
        const double ick = okk ? rsqrt(gkk) : 1.0;
        for (int i = k + 1 + threadIdx.x; i < pd; i += blockDim.x) J[i + (size_t)k * pd] *= ick;
        if (threadIdx.x == 0) {
          cn0[k] = ick;
          if (!okk) s_bad = 1;
        }
        __syncthreads();
        for (int j = k + 1 + w; j < pd; j += nw) {
          const double cj = J[j + (size_t)k * pd];
          for (int i = j + lane; i < pd; i += 32) J[i + (size_t)j * pd] = fma(-J[i + (size_t)k * pd], cj, J[i + (size_t)j * pd]);
        }
        __syncthreads();
      }
      // Q C^T = V0 by forward substitution along each row, one thread per row
      // (four partial sums shorten the FP64 dependency chain)
      if (!s_bad)
        for (int r = threadIdx.x; r < pd; r += blockDim.x)
          for (int c = 0; c < pd; ++c) {
            double s0 = Tg[r + (size_t)c * pd], s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int j = 0;
            for (; j + 3 < c; j += 4) {
              s0 = fma(-Tg[r + (size_t)j * pd], J[c + (size_t)j * pd], s0);
              s1 = fma(-Tg[r + (size_t)(j + 1) * pd], J[c + (size_t)(j + 1) * pd], s1);
              s2 = fma(-Tg[r + (size_t)(j + 2) * pd], J[c + (size_t)(j + 2) * pd], s2);
              s3 = fma(-Tg[r + (size_t)(j + 3) * pd], J[c + (size_t)(j + 3) * pd], s3);
            }
            for (; j < c; ++j) s0 = fma(-Tg[r + (size_t)j * pd], J[c + (size_t)j * pd], s0);
            Tg[r + (size_t)c * pd] = ((s0 + s1) + (s2 + s3)) * cn0[c];
          }
      __syncthreads();
      // no usable pre-rotation: V0 = I and L stays as it is
      for (int t = threadIdx.x; t < pd * pd; t += blockDim.x)
        J[t] = s_bad ? (((t % pd) == (t / pd)) ? 1.0 : 0.0) : Tg[t];
      __syncthreads();
    }
    for (int t = threadIdx.x; t < p * pd; t += blockDim.x) {  // T = L V0
      const int r = t % p, b = t / p;
      double u = 0.0;
      for (int a = 0; a < pd; ++a) u = fma(A[r + (size_t)a * p], J[a + (size_t)b * pd], u);
      Tg[t] = u;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < p * pd; t += blockDim.x) A[t] = Tg[t];
    __syncthreads();
  }
  const double eps = DBL_EPSILON * p, eps2 = eps * eps;
  // ---- 2b. FP64 sweeps.  In a cluster, CTA `me` takes the pairs
  // [plo, phi) of every round and writes the two columns of A and V it
  // rotates, and their norms, into every other CTA's shared memory, so that
  // all CTAs hold the same A, V and norms after each round's cluster
  // barrier; every pair sees the same inputs as in one CTA, so the result
  // is bit-identical to the single-CTA kernel.
  const int npairs = q / 2;
  const int plo = (int)((long)npairs * me / cl), phi = (int)((long)npairs * (me + 1) / cl);
  // stores of a value into the same shared-memory slot of every CTA
  auto put_all = [&](double* slot, double v) {
    if (cl == 1) {
      *slot = v;
    } else {
      cg::cluster_group cluster = cg::this_cluster();
      for (int cc = 0; cc < cl; ++cc) *cluster.map_shared_rank(slot, cc) = v;
    }
  };
  auto csync = [&] {
    if (cl > 1)
      cg::this_cluster().sync();
    else
      __syncthreads();
  };
  csync();  // every CTA is running before its shared memory is written
  int sweep = 0;
  for (; sweep < SVD_MAX_SWEEPS && pd > 1; ++sweep) {
    // exact squared column norms at the start of the sweep; inside the sweep
    // each rotation updates them as alpha - t gamma, beta + t gamma
    for (int j = w; j < pd; j += nw) {
      double sq = 0.0;
      for (int r = lane; r < p; r += 32) sq = fma(A[r + (size_t)j * p], A[r + (size_t)j * p], sq);
      sq = warp_sum(sq);
      if (lane == 0) cn[j] = sq;
    }
    if (threadIdx.x == 0) {
      s_rot = 0;
      s_tmax = 0;
    }
    // in a cluster, no CTA updates another's norms before that one has
    // computed them
    csync();
    for (int step = 0; step < q - 1; ++step) {
      // (a) H lanes per pair: the off-diagonal g = <c_i, c_j>
      for (int base = plo + w * PW; base < phi; base += nw * PW) {
        const int pr = base + lane / H;
        int i = 0, j = 0;
        bool ok = pr < phi;
        if (ok) {
          i = (pr == 0) ? 0 : 1 + ((pr - 1 + step) % (q - 1));
          j = 1 + ((q - 1 - pr - 1 + step) % (q - 1));
          ok = i < pd && j < pd;
        }
        double ga = 0.0;
        if (ok) {
          const double* ci = A + (size_t)i * p;
          const double* cj = A + (size_t)j * p;
          for (int r = sub; r < p; r += H) ga = fma(ci[r], cj[r], ga);
        }
        ga = group_sum(ga, H);
        if (ok && sub == 0) gam[pr] = ga;
      }
      __syncthreads();
      // (b) warp 0, one lane per pair: the rotations of the whole round (an
      // FP64 instruction costs its SMSP the same with 1 or 32 active lanes)
      if (w == 0) {
        for (int pr = plo + lane; pr < phi; pr += 32) {
          const int i = (pr == 0) ? 0 : 1 + ((pr - 1 + step) % (q - 1));
          const int j = 1 + ((q - 1 - pr - 1 + step) % (q - 1));
          double c = 1.0, sn = 0.0;
          if (i < pd && j < pd) {
            const double ga = gam[pr], al = cn[i], be = cn[j];
            // |ga| <= eps sqrt(al be), compared in squares (no FP64 roots)
            if (!(al <= thr || be <= thr || ga * ga <= eps2 * al * be)) {
              // The angle only steers convergence: it is formed in FP32 from
              // dd and ga scaled by the same power of two (exact; the larger
              // lands in [1, 2)), while c = 1/sqrt(1 + t^2) in FP64 keeps the
              // applied rotation orthogonal to FP64 accuracy (no FP64 square
              // root or division per rotation).
              const double dd = be - al;
              const unsigned long long ebits = __double_as_longlong(fmax(fabs(dd), fabs(ga)));
              const int ex = (int)((ebits >> 52) & 0x7FF);
              const double sc = __longlong_as_double((unsigned long long)(2046 - min(ex, 2045)) << 52);
              const float dds = (float)(dd * sc), gas = (float)(ga * sc);
              const float tf =
                  (dds >= 0.0f ? 2.0f * gas : -2.0f * gas) / (fabsf(dds) + sqrtf(fmaf(dds, dds, 4.0f * gas * gas)));
              double t = (double)tf;
              if (!(fabsf(tf) > 0.0f && isfinite(tf)))  // FP64 formula where FP32 cannot resolve the angle
                t = (dd >= 0.0 ? 2.0 * ga : -2.0 * ga) / (fabs(dd) + sqrt(fma(dd, dd, 4.0 * ga * ga)));
              c = rsqrt(fma(t, t, 1.0));
              sn = c * t;
              const double ni = fma(-t, ga, al), nj = fma(t, ga, be);
              put_all(&cn[i], ni);
              put_all(&cn[j], nj);
              // |t| as its float bit pattern: non-negative floats order like ints
              atomicMax(&s_tmax, __float_as_int(fminf((float)fabs(t), 1.0f)));
              s_rot = 1;
            }
          }
          rc_c[pr] = c;
          rc_s[pr] = sn;
        }
      }
      __syncthreads();
      // (c) H lanes per pair: apply the rotation to L and V (no shuffles:
      // the lanes of a pair go their own way), in every CTA of the cluster
      for (int pr = plo + w * PW + lane / H; pr < phi; pr += nw * PW) {
        const double sn = rc_s[pr];
        if (sn == 0.0) continue;
        const double c = rc_c[pr];
        const int i = (pr == 0) ? 0 : 1 + ((pr - 1 + step) % (q - 1));
        const int j = 1 + ((q - 1 - pr - 1 + step) % (q - 1));
        for (int r = sub; r < p; r += H) {
          const double x = A[r + (size_t)i * p], y = A[r + (size_t)j * p];
          const double nx = c * x - sn * y, ny = sn * x + c * y;
          put_all(&A[r + (size_t)i * p], nx);
          put_all(&A[r + (size_t)j * p], ny);
        }
        for (int r = sub; r < pd; r += H) {
          const double x = J[r + (size_t)i * pd], y = J[r + (size_t)j * pd];
          const double nx = c * x - sn * y, ny = sn * x + c * y;
          put_all(&J[r + (size_t)i * pd], nx);
          put_all(&J[r + (size_t)j * pd], ny);
        }
      }
      csync();
    }
    // the sweep's outcome over the cluster: every CTA reads every CTA's
    // flags, then waits until all have read them before they are reset
    int rot = s_rot, tmax = s_tmax;
    if (cl > 1) {
      cg::cluster_group cluster = cg::this_cluster();
      for (int cc = 0; cc < cl; ++cc) {
        rot |= *cluster.map_shared_rank(&s_rot, cc);
        tmax = max(tmax, *cluster.map_shared_rank(&s_tmax, cc));
      }
      cluster.sync();
    }
    if (rot == 0) break;
    // every rotation of this sweep was below 1e-7: quadratic convergence puts
    // the remaining off-diagonal at ~1e-14 relative, so the confirming sweep
    // (which would rotate nothing above the threshold) is skipped
    if (__int_as_float(tmax) < 1e-7f) {
      ++sweep;
      break;
    }
    __syncthreads();
  }
  // the rest runs in CTA 0 alone (no shared memory of another CTA is touched
  // after the last cluster barrier)
  if (me != 0) return;
  // ---- 3. singular values, order, truncation
  for (int j = w; j < pd; j += nw) {
    double s = 0.0;
    for (int r = lane; r < p; r += 32) s = fma(A[r + (size_t)j * p], A[r + (size_t)j * p], s);
    s = warp_sum(s);
    if (lane == 0) cn[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < pd; j += blockDim.x) {
    // ranking by (value desc, index asc) with non-finite values mapped to -1,
    // a strict total order, so order[] is always a permutation of 0..pd-1
    const double vj = isfinite(cn[j]) ? cn[j] : -1.0;
    int rk = 0;
    for (int l = 0; l < pd; ++l) {
      const double vl = isfinite(cn[l]) ? cn[l] : -1.0;
      rk += (vl > vj) || (vl == vj && l < j);
    }
    order[rk] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double bound = tol * tol * fro2;
    double tail = qr_tail2;
    int k = pd;
    for (int c = pd - 1; c >= 0; --c) {
      const double sv = cn[order[c]];
      const double nt = fma(sv, sv, tail);
      if (nt <= bound) {
        tail = nt;
        k = c;
      } else {
        break;
      }
    }
    if (k < 1) k = 1;
    if (k > cap) k = cap;
    double dis = qr_tail2;
    for (int c = pd - 1; c >= k; --c) dis = fma(cn[order[c]], cn[order[c]], dis);
    for (int c = 0; c < p; ++c) sig[c] = c < pd ? cn[order[c]] : 0.0;
    s_k = k;
    info[0] = k;
    info[1] = pd;
    info[2] = sweep + 1;
    tail_out[0] = sqrt(dis);
    tail_out[1] = sqrt(fro2);
    if (sweep >= SVD_MAX_SWEEPS) atomicOr(status, DEV_JACOBI_NOCONV);
  }
  __syncthreads();
  const int k = s_k;
  // US = P (L V): row piv[r] of US is row r of L V
  for (int t = threadIdx.x; t < p * k; t += blockDim.x) {
    const int r = t % p, c = t / p;
    US[piv[r] + (size_t)c * p] = c < pd ? A[r + (size_t)order[c] * p] : 0.0;
  }
  // Vout = Q [V; 0]: reflectors applied last-to-first to Z (p x k in
  // shared memory, row-major with an odd row length).  Each warp owns Cq
  // columns of Z and, per column, the rows i = rq (mod Kq) (lane (rq, cq) =
  // (lane / Cq, lane mod Cq)); a reflector's inner products are finished by
  // shuffles and no block barrier is needed, the reflectors and their
  // factors being first copied into shared memory.
  __syncthreads();  // A (L V) has been read into US: reuse it for Z
  const int kz = (k < p) ? (k | 1) : k;  // Z must fit in A's p x p doubles
  double* Z = A;                          // p x kz
  for (int t = threadIdx.x; t < p * k; t += blockDim.x) {
    const int r = t / k, c = t % k;
    Z[(size_t)r * kz + c] = (c < pd && r < pd) ? J[r + (size_t)order[c] * pd] : ((c >= pd && r == c) ? 1.0 : 0.0);
  }
  __syncthreads();  // J (V) has been read into Z: reuse it for the reflectors
  double* hvs = J;  // p x pd, column kk holds reflector kk below row kk
  for (int t = threadIdx.x; t < p * pd; t += blockDim.x) hvs[t] = HV[t];
  for (int t = threadIdx.x; t < pd; t += blockDim.x) cn0[t] = htau[t];
  __syncthreads();
  {
    // lanes per column: the fewest FP64 instructions on the busiest SM
    // sub-partition over the pd reflectors (rows kk..p-1, p/2 on average)
    int Kq = 32;
    long bestq = 0x7fffffffffffffffL;
    for (int kq = 2; kq <= 32; kq <<= 1) {
      const int cpw = 32 / kq, warps = (k + cpw - 1) / cpw;
      if (warps > nw) continue;
      int lg = 0;
      while ((1 << lg) < kq) ++lg;
      const long cost = (long)((warps + 3) / 4) * (2L * ((p / 2 + kq - 1) / kq) + lg + 3);
      if (cost < bestq) {
        bestq = cost;
        Kq = kq;
      }
    }
    const int Cq = 32 / Kq, rq = lane / Cq, cq = lane % Cq, c = w * Cq + cq;
    if (w * Cq < k) {  // warp-uniform
      const bool colv = c < k;
      for (int kk = pd - 1; kk >= 0; --kk) {
        const double tk = cn0[kk];
        if (tk == 0.0) continue;
        const double* hv = hvs + (size_t)kk * p;
        const bool top = rq == (kk & (Kq - 1));
        const int i0 = kk + 1 + ((rq - kk - 1) & (Kq - 1));
        double d = 0.0;
        if (colv) {
          if (top) d = Z[(size_t)kk * kz + c];
          for (int i = i0; i < p; i += Kq) d = fma(hv[i], Z[(size_t)i * kz + c], d);
        }
        for (int o = Cq; o < 32; o <<= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        d *= tk;
        if (colv) {
          if (top) Z[(size_t)kk * kz + c] -= d;
          for (int i = i0; i < p; i += Kq) Z[(size_t)i * kz + c] = fma(-d, hv[i], Z[(size_t)i * kz + c]);
        }
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * k; t += blockDim.x) {
    const int r = t % p, c = t / p;
    Vout[r + (size_t)c * p] = Z[(size_t)r * kz + c];
  }
}

// CTAs that share a p x p SVD's FP64 sweeps: each takes 1/cl of a round's
// pairs for one cluster barrier per round, which pays where a round's work
// (p/2 pairs of ~9p FP64 operations) is well above the barrier's cost
// (p = 68: 2.8 -> 2.0 ms, p = 112: 9.5 -> 5.9 ms).  Used where the Exec allows
// it (the standalone entry points, not the solver's stages).  TT_SVD_CLUSTER
// (environment, read once): 0 or 1 keeps one CTA, 2, 4 or 8 sets the size from
// p = 48 up.
static int svd_cluster_size(int p) {
  static const int forced = [] {
    const char* e = std::getenv("TT_SVD_CLUSTER");
    return e ? std::atoi(e) : -1;
  }();
  if (forced >= 0) return (forced == 2 || forced == 4 || forced == 8) && p >= 48 ? forced : 1;
  return p >= 96 ? 8 : p >= 48 ? 4 : 1;
}

static bool svd_cluster_ok(int cl) {
  static int ok[SVD_MAX_CLUSTER + 1] = {};  // 0 unknown, 1 yes, 2 no
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (ok[cl] == 0) {
    ok[cl] = 2;
    if (smem_attr_once_impl(reinterpret_cast<const void*>(k_svd_small)) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(SVD_THREADS);
      cfg.dynamicSmemBytes = 2 * (size_t)112 * 112 * 8;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_svd_small, &cfg) == cudaSuccess && nc > 0) ok[cl] = 1;
      (void)cudaGetLastError();
    }
  }
  return ok[cl] == 1;
}

void jacobi_svd(Exec& ex, const double* M, int p, double tol, int cap, double* US, double* V, double* sig,
                int* k_out, double* tail_out) {
  TT_REQUIRE(p >= 1 && p <= 112, TT_ERR_ARG);
  Scope sc(*ex.ar);
  // scratch for the cluster size of p whatever the device supports, so that
  // the sizing pass needs no device
  const int cl_want = svd_cluster_size(p);
  double* scr = ex.ar->get<double>((size_t)cl_want * svd_scratch_doubles(p));
  if (ex.dry) return;
  const size_t smem = 2 * (size_t)p * p * 8;
  smem_attr_once(k_svd_small);
  const int cl = (cl_want > 1 && ex.svd_cluster && svd_cluster_ok(cl_want)) ? cl_want : 1;
  // deflation level: far below the truncation tolerance and the 1e-10 parity
  // bar on the FP64 path; the precision forms' cores carry FP32 round-off
  // (~1e-7 relative), so there it deflates at 1e-2 of their tolerance
  const double defl = ex.precision == TT_FP64 ? std::max(std::min(1e-13, 1e-2 * tol), 1e-15)
                                              : std::max(1e-2 * tol, 1e-13);
  // algorithmic work: pivoted QR (4/3 p^3) plus a nominal 3 Jacobi sweeps
  const double fl = 4.0 / 3.0 * p * (double)p * p + 3.0 * (p * (p - 1) / 2.0) * 18.0 * p;
  if (cl > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(SVD_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ex.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TT_KERNEL(ex, K_JACOBI, fl, 8.0 * 4.0 * p * (double)p,
              TT_CUDA(cudaLaunchKernelEx(&cfg, k_svd_small, M, p, tol, cap, defl, US, V, sig, k_out, tail_out, scr,
                                         ex.dev_status)));
    return;
  }
  TT_KERNEL(ex, K_JACOBI, fl, 8.0 * 4.0 * p * (double)p,
            k_svd_small<<<1, SVD_THREADS, smem, ex.s>>>(M, p, tol, cap, defl, US, V, sig, k_out, tail_out, scr,
                                                        ex.dev_status));
}

// ============================================================== maxvol
constexpr int MV_THREADS = 1024;

struct ArgMax {
  double v;
  long idx;
};
__device__ __forceinline__ ArgMax amax_better(ArgMax a, ArgMax b) {
  // larger value wins; ties go to the smaller index
  if (b.v > a.v || (b.v == a.v && b.idx < a.idx)) return b;
  return a;
}
__device__ ArgMax block_argmax(ArgMax x, double* rv, long* ri) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ArgMax y{__shfl_xor_sync(0xffffffffu, x.v, o), __shfl_xor_sync(0xffffffffu, x.idx, o)};
    x = amax_better(x, y);
  }
  __syncthreads();
  if (lane == 0) {
    rv[w] = x.v;
    ri[w] = x.idx;
  }
  __syncthreads();
  if (w == 0) {
    ArgMax y{lane < nw ? rv[lane] : -1.0, lane < nw ? ri[lane] : 0x7fffffffffffffffL};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ArgMax z{__shfl_xor_sync(0xffffffffu, y.v, o), __shfl_xor_sync(0xffffffffu, y.idx, o)};
      y = amax_better(y, z);
    }
    if (lane == 0) {
      rv[32] = y.v;
      ri[32] = y.idx;
    }
  }
  __syncthreads();
  return ArgMax{rv[32], ri[32]};
}

// W: n x r scratch (copy of U), B: n x r scratch, P: r x r scratch, all in
// the working type T (U itself is FP64).  The kernel only chooses row
// indices: every decision is a comparison of magnitudes (the largest pivot,
// |B_ij| against 1 + delta with delta = 1e-2), which FP32 resolves, so the
// solver runs it in FP32, an instruction that costs 1/64 of an FP64 one on
// this GPU; the skeleton built from the chosen rows is FP64.
template <typename T>
__global__ void __launch_bounds__(MV_THREADS) k_maxvol(const double* __restrict__ U, int n, int r, double delta,
                                                      int max_iter, T* W, T* B, T* P, int* I, unsigned* status) {
  __shared__ double rv[33];
  __shared__ long ri[33];
  __shared__ int piv[128];
  __shared__ double s_inv;
  extern __shared__ unsigned char freeflag[];  // n bytes
  for (long t = threadIdx.x; t < (long)n * r; t += blockDim.x) W[t] = T(U[t]);
  for (int i = threadIdx.x; i < n; i += blockDim.x) freeflag[i] = 1;
  __syncthreads();
  // 1. partial-pivoting row choice, rows left in place
  for (int k = 0; k < r; ++k) {
    ArgMax best{-1.0, 0x7fffffffffffffffL};
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (freeflag[i]) {
        // a NaN entry counts as 0 (and is flagged), so a free row is always chosen
        double v = fabs((double)W[i + (size_t)k * n]);
        if (!(v >= 0.0)) {
          v = 0.0;
          atomicOr(status, DEV_NONFINITE);
        }
        best = amax_better(best, ArgMax{v, (long)i});
      }
    best = block_argmax(best, rv, ri);
    const int pr = (int)best.idx;
    if (threadIdx.x == 0) {
      piv[k] = pr;
      freeflag[pr] = 0;
    }
    __syncthreads();
    const T pv = W[pr + (size_t)k * n];
    if (threadIdx.x == 0) s_inv = pv != T(0) ? 1.0 / (double)pv : 0.0;
    __syncthreads();
    const T ipv = T(s_inv);
    if (pv != T(0) && k + 1 < r) {
      // column k is read only (it is not used again), columns k+1.. updated
      for (long t = threadIdx.x; t < (long)n * (r - k - 1); t += blockDim.x) {
        const int i = int(t % n), c = k + 1 + int(t / n);
        if (freeflag[i]) {
          const T f = W[i + (size_t)k * n] * ipv;
          W[i + (size_t)c * n] = fma(-f, W[pr + (size_t)c * n], W[i + (size_t)c * n]);
        }
      }
    }
    __syncthreads();
  }
  // 2. B = U P^{-1} with P = U[piv, :]: Gauss-Jordan on [P | I] in P (r x 2r)
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    const int i = t % r, j = t / r;
    P[i + (size_t)j * r] = T(U[piv[i] + (size_t)j * n]);
    P[i + (size_t)(j + r) * r] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  // Solve X P = U for X = B: equivalently P^T X^T = U^T.  Invert P by
  // Gauss-Jordan with partial pivoting (row swaps recorded in the matrix).
  __shared__ int gpiv;
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      int best = k;
      double bv = fabs((double)P[k + (size_t)k * r]);
      for (int i = k + 1; i < r; ++i) {
        const double v = fabs((double)P[i + (size_t)k * r]);
        if (v > bv) {
          bv = v;
          best = i;
        }
      }
      gpiv = best;
    }
    __syncthreads();
    const int pr = gpiv;
    if (pr != k)
      for (int c = threadIdx.x; c < 2 * r; c += blockDim.x) {
        const T a = P[k + (size_t)c * r];
        P[k + (size_t)c * r] = P[pr + (size_t)c * r];
        P[pr + (size_t)c * r] = a;
      }
    __syncthreads();
    const T d = P[k + (size_t)k * r];
    if (threadIdx.x == 0) s_inv = d != T(0) ? 1.0 / (double)d : 0.0;
    __syncthreads();
    const T invd = T(s_inv);
    if (d != T(0)) {
      for (int c = threadIdx.x; c < 2 * r; c += blockDim.x) P[k + (size_t)c * r] *= invd;
    }
    __syncthreads();
    for (long t = threadIdx.x; t < (long)r * 2 * r; t += blockDim.x) {
      const int i = int(t % r), c = int(t / r);
      if (i != k) {
        const T f = P[i + (size_t)k * r];
        if (c != k) P[i + (size_t)c * r] = fma(-f, P[k + (size_t)c * r], P[i + (size_t)c * r]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      if (i != k) P[i + (size_t)k * r] = T(0);
    __syncthreads();
  }
  // Pinv = P[:, r:2r];  B = U Pinv (n x r)
  for (long t = threadIdx.x; t < (long)n * r; t += blockDim.x) {
    const int i = int(t % n), j = int(t / n);
    T s = T(0);
    for (int l = 0; l < r; ++l) s = fma(T(U[i + (size_t)l * n]), P[l + (size_t)(j + r) * r], s);
    B[t] = s;
  }
  for (int k = threadIdx.x; k < r; k += blockDim.x) I[k] = piv[k];
  __syncthreads();
  // 3. swap rows while some |B_ij| > 1 + delta (ties: smallest i*r + j)
  int it = 0;
  for (; it < max_iter; ++it) {
    ArgMax best{-1.0, 0x7fffffffffffffffL};
    for (long t = threadIdx.x; t < (long)n * r; t += blockDim.x) {
      const int i = int(t % n), j = int(t / n);
      best = amax_better(best, ArgMax{fabs((double)B[t]), (long)i * r + j});
    }
    best = block_argmax(best, rv, ri);
    if (best.v <= 1.0 + delta) break;
    const int bi = int(best.idx / r), bj = int(best.idx % r);
    if (threadIdx.x == 0) s_inv = 1.0 / (double)B[bi + (size_t)bj * n];
    // B -= B[:, j] (B[i, :] - e_j)^T / pivot ; use W as scratch for the column and row
    for (int i = threadIdx.x; i < n; i += blockDim.x) W[i] = B[i + (size_t)bj * n];
    for (int j = threadIdx.x; j < r; j += blockDim.x) W[n + j] = B[bi + (size_t)j * n] - (j == bj ? T(1) : T(0));
    __syncthreads();
    const T ipiv = T(s_inv);
    for (long t = threadIdx.x; t < (long)n * r; t += blockDim.x) {
      const int i = int(t % n), j = int(t / n);
      B[t] = fma(-W[i] * ipiv, W[n + j], B[t]);
    }
    if (threadIdx.x == 0) I[bj] = bi;
    __syncthreads();
  }
  if (threadIdx.x == 0 && it >= max_iter) atomicOr(status, DEV_MAXVOL_NOCONV);
}

// ---------------------------------------------------------------- maxvol over a cluster
// The same three phases as k_maxvol with the n rows split over the CTAs of a
// thread-block cluster, each CTA keeping its rows of the working matrix (FP32,
// row-major) in its own shared memory: the single-CTA kernel streams the whole
// n x r matrix through one SM's L2 path on every pivot step, the cluster
// scans shared memory on up to 8 SMs.  Per pivot step each CTA publishes its
// best local candidate and a copy of that row in a double-buffered slot, one
// cluster barrier makes the slots visible, and every CTA reads all slots
// through distributed shared memory and takes the same (largest value,
// smallest index) decision, so all CTAs run the same number of steps and
// barriers.  The r x r inverse is formed redundantly (identically) by every
// CTA.  Row choices and tie rules are those of k_maxvol.
constexpr int MVC_THREADS = 512;
constexpr int MVC_MAX_CLUSTER = 8;

struct MvcLayout {
  int nc;  // rows per CTA
  size_t off_flag, off_col, off_prow, off_P, off_slot, bytes;
  int slot_floats;  // per slot: value, index (as bits), row of r values
};
__host__ __device__ inline MvcLayout mvc_layout(int n, int r, int cl) {
  MvcLayout L;
  L.nc = (n + cl - 1) / cl;
  size_t o = (size_t)L.nc * r * 4;  // rows
  L.off_col = o;
  o += (size_t)L.nc * 4;  // saved pivot column (phase 3)
  L.off_prow = o;
  o += (size_t)r * 4;  // pivot row
  L.off_P = o;
  o += (size_t)2 * r * r * 4;  // [P | I] for Gauss-Jordan
  L.off_slot = o;
  L.slot_floats = 2 + r;
  o += (size_t)2 * L.slot_floats * 4;  // two candidate slots
  L.off_flag = o;
  o += (size_t)L.nc;  // free-row flags
  L.bytes = (o + 15) & ~(size_t)15;
  return L;
}

__device__ __forceinline__ bool mv_better(float v, long idx, float bv, long bidx) {
  return v > bv || (v == bv && idx < bidx);
}

__global__ void __launch_bounds__(MVC_THREADS) k_maxvol_cluster(const double* __restrict__ U, int n, int r,
                                                                double delta, int max_iter, int* I,
                                                                unsigned* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int cl = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smraw[];
  const MvcLayout L = mvc_layout(n, r, cl);
  float* W = reinterpret_cast<float*>(smraw);  // nc x r, row-major
  float* col = reinterpret_cast<float*>(smraw + L.off_col);
  float* prow = reinterpret_cast<float*>(smraw + L.off_prow);
  float* P = reinterpret_cast<float*>(smraw + L.off_P);  // r x 2r, column-major
  float* slot = reinterpret_cast<float*>(smraw + L.off_slot);
  unsigned char* freeflag = smraw + L.off_flag;
  __shared__ double rv[33];
  __shared__ long ri[33];
  __shared__ int piv[128];
  __shared__ int s_win, s_gp;
  __shared__ float s_inv;
  const int row0 = me * L.nc, nloc = max(0, min(L.nc, n - row0));
  for (int t = threadIdx.x; t < nloc * r; t += blockDim.x) {
    const int i = t / r, j = t - i * r;
    W[t] = (float)U[(size_t)(row0 + i) + (size_t)j * n];
  }
  for (int i = threadIdx.x; i < L.nc; i += blockDim.x) freeflag[i] = 1;
  __syncthreads();
  // publish this CTA's candidate (value, global index, a copy of local row
  // li) in slot buffer b; li < 0: no candidate
  auto publish = [&](int b, float v, long gidx, int li) {
    float* s = slot + (size_t)b * L.slot_floats;
    if (threadIdx.x == 0) {
      s[0] = v;
      reinterpret_cast<int*>(s)[1] = (int)gidx;
    }
    if (li >= 0)
      for (int j = threadIdx.x; j < r; j += blockDim.x) s[2 + j] = W[(size_t)li * r + j];
  };
  // after the cluster barrier: the winning slot's CTA (s_win) and index (s_gp)
  auto decide = [&](int b) {
    if (threadIdx.x == 0) {
      float bv = -2.0f;
      long bi = 0x7fffffffffffffffL;
      int win = 0;
      for (int q = 0; q < cl; ++q) {
        const float* rs = cluster.map_shared_rank(slot + (size_t)b * L.slot_floats, q);
        const float v = rs[0];
        const long idx = reinterpret_cast<const int*>(rs)[1];
        if (mv_better(v, idx, bv, bi)) {
          bv = v;
          bi = idx;
          win = q;
        }
      }
      s_win = win;
      s_gp = (int)bi;
    }
    __syncthreads();
  };
  // 1. partial-pivoting row choice
  for (int k = 0; k < r; ++k) {
    ArgMax best{-1.0, 0x7fffffffffffffffL};
    for (int i = threadIdx.x; i < nloc; i += blockDim.x)
      if (freeflag[i]) {
        double v = fabs((double)W[(size_t)i * r + k]);
        if (!(v >= 0.0)) {
          v = 0.0;
          atomicOr(status, DEV_NONFINITE);
        }
        best = amax_better(best, ArgMax{v, (long)i});
      }
    best = block_argmax(best, rv, ri);
    const int li = best.v >= 0.0 ? (int)best.idx : -1;
    const int sb = k & 1;  // slot of publication number k
    publish(sb, li >= 0 ? (float)best.v : -1.0f, li >= 0 ? (long)(row0 + li) : 0x7fffffffL, li);
    cluster.sync();
    decide(sb);
    const int win = s_win, pr = s_gp;
    {
      const float* rs = cluster.map_shared_rank(slot + (size_t)sb * L.slot_floats, win);
      for (int j = threadIdx.x; j < r; j += blockDim.x) prow[j] = rs[2 + j];
    }
    if (threadIdx.x == 0) {
      piv[k] = pr;
      if (win == me) freeflag[pr - row0] = 0;
    }
    __syncthreads();
    const float pv = prow[k];
    if (pv != 0.0f && k + 1 < r) {
      const float ipv = (float)(1.0 / (double)pv);
      const int w = r - k - 1;
      for (int t = threadIdx.x; t < nloc * w; t += blockDim.x) {
        const int i = t / w, c = k + 1 + (t - i * w);
        if (freeflag[i]) {
          const float f = W[(size_t)i * r + k] * ipv;
          W[(size_t)i * r + c] = fmaf(-f, prow[c], W[(size_t)i * r + c]);
        }
      }
    }
    __syncthreads();
  }
  // 2. B = U P^{-1}, P = U[piv, :]: Gauss-Jordan on [P | I] (every CTA)
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
    const int i = t % r, j = t / r;
    P[i + (size_t)j * r] = (float)U[piv[i] + (size_t)j * n];
    P[i + (size_t)(j + r) * r] = (i == j) ? 1.0f : 0.0f;
  }
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (threadIdx.x == 0) {
      int bsel = k;
      double bv = fabs((double)P[k + (size_t)k * r]);
      for (int i = k + 1; i < r; ++i) {
        const double v = fabs((double)P[i + (size_t)k * r]);
        if (v > bv) {
          bv = v;
          bsel = i;
        }
      }
      s_gp = bsel;
    }
    __syncthreads();
    const int pr = s_gp;
    if (pr != k)
      for (int c = threadIdx.x; c < 2 * r; c += blockDim.x) {
        const float a = P[k + (size_t)c * r];
        P[k + (size_t)c * r] = P[pr + (size_t)c * r];
        P[pr + (size_t)c * r] = a;
      }
    __syncthreads();
    const float d = P[k + (size_t)k * r];
    if (threadIdx.x == 0) s_inv = d != 0.0f ? (float)(1.0 / (double)d) : 0.0f;
    __syncthreads();
    if (d != 0.0f)
      for (int c = threadIdx.x; c < 2 * r; c += blockDim.x) P[k + (size_t)c * r] *= s_inv;
    __syncthreads();
    for (int t = threadIdx.x; t < r * 2 * r; t += blockDim.x) {
      const int i = t % r, c = t / r;
      if (i != k && c != k)
        P[i + (size_t)c * r] = fmaf(-P[i + (size_t)k * r], P[k + (size_t)c * r], P[i + (size_t)c * r]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      if (i != k) P[i + (size_t)k * r] = 0.0f;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nloc * r; t += blockDim.x) {
    const int i = t / r, j = t - i * r;
    float s = 0.0f;
    for (int l = 0; l < r; ++l) s = fmaf((float)U[(size_t)(row0 + i) + (size_t)l * n], P[l + (size_t)(j + r) * r], s);
    W[t] = s;
  }
  __syncthreads();
  // 3. swap rows while some |B_ij| > 1 + delta (ties: smallest i r + j)
  int it = 0;
  for (; it < max_iter; ++it) {
    ArgMax best{-1.0, 0x7fffffffffffffffL};
    for (int t = threadIdx.x; t < nloc * r; t += blockDim.x) {
      const int i = t / r, j = t - i * r;
      best = amax_better(best, ArgMax{fabs((double)W[t]), (long)(row0 + i) * r + j});
    }
    best = block_argmax(best, rv, ri);
    const int li = best.v >= 0.0 ? (int)(best.idx / r) - row0 : -1;
    // publications continue the numbering of phase 1 (r of them), so two
    // uses of one slot are always a cluster barrier apart
    const int sb = (r + it) & 1;
    publish(sb, li >= 0 ? (float)best.v : -1.0f, li >= 0 ? best.idx : 0x7fffffffL, li);
    cluster.sync();
    decide(sb);
    const int win = s_win, gidx = s_gp;
    {
      const float* rs = cluster.map_shared_rank(slot + (size_t)sb * L.slot_floats, win);
      if (threadIdx.x == 0) s_inv = rs[0];
      for (int j = threadIdx.x; j < r; j += blockDim.x) prow[j] = rs[2 + j];
    }
    __syncthreads();
    if ((double)s_inv <= 1.0 + delta) break;  // the same decision in every CTA
    const int bi = gidx / r, bj = gidx - bi * r;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) col[i] = W[(size_t)i * r + bj];
    __syncthreads();
    const float ipiv = (float)(1.0 / (double)prow[bj]);
    for (int t = threadIdx.x; t < nloc * r; t += blockDim.x) {
      const int i = t / r, j = t - i * r;
      const float rj = prow[j] - (j == bj ? 1.0f : 0.0f);
      W[t] = fmaf(-col[i] * ipiv, rj, W[t]);
    }
    if (threadIdx.x == 0) piv[bj] = bi;
    __syncthreads();
  }
  if (me == 0) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) I[k] = piv[k];
    if (threadIdx.x == 0 && it >= max_iter) atomicOr(status, DEV_MAXVOL_NOCONV);
  }
  // no CTA leaves while another may still read its slots
  cluster.sync();
}

// whether an 8-CTA cluster of k_maxvol_cluster with the shared-memory budget
// can be resident on this device (checked once per process)
static bool maxvol_cluster_ok() {
  static const bool ok = [] {
    if (smem_attr_once_impl(reinterpret_cast<const void*>(k_maxvol_cluster)) != cudaSuccess) return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(MVC_MAX_CLUSTER);
    cfg.blockDim = dim3(MVC_THREADS);
    cfg.dynamicSmemBytes = QR_SMEM_MAX;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = MVC_MAX_CLUSTER;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&nc, k_maxvol_cluster, &cfg);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return false;
    }
    return nc > 0;
  }();
  return ok;
}

void maxvol(Exec& ex, const double* U, int n, int r, double delta, int max_iter, int* I) {
  TT_REQUIRE(r >= 1 && r <= 128 && n >= r, TT_ERR_ARG);
  using T = float;
  Scope sc(*ex.ar);
  T* W = ex.ar->get<T>((size_t)n * r + n + r);
  T* B = ex.ar->get<T>((size_t)n * r);
  T* P = ex.ar->get<T>((size_t)2 * r * r);
  if (ex.dry) return;
  // cluster form: the smallest power-of-two cluster (at most 8 CTAs) that
  // leaves each CTA at most 8192 entries, when it fits shared memory;
  // TT_MAXVOL_CLUSTER=0 (environment, read once) keeps the single-CTA
  // kernel, which makes the same choices (tests compare the two)
  static const bool allow = [] {
    const char* e = std::getenv("TT_MAXVOL_CLUSTER");
    return !(e && std::atoi(e) == 0);
  }();
  int cl = 1;
  while (cl < MVC_MAX_CLUSTER && (long)ceil_div(n, cl) * r > 8192) cl *= 2;
  const MvcLayout L = mvc_layout(n, r, cl);
  if (allow && r <= 128 && L.bytes <= QR_SMEM_MAX && maxvol_cluster_ok()) {
    smem_attr_once(k_maxvol_cluster);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(MVC_THREADS);
    cfg.dynamicSmemBytes = L.bytes;
    cfg.stream = ex.s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TT_KERNEL(ex, K_MAXVOL, 3.0 * n * (double)r * r, (8.0 + 2.0 * sizeof(T)) * n * (double)r,
              TT_CUDA(cudaLaunchKernelEx(&cfg, k_maxvol_cluster, U, n, r, delta, max_iter, I, ex.dev_status)));
    return;
  }
  const size_t smem = (size_t)n;
  TT_REQUIRE(smem <= 200 * 1024, TT_ERR_ARG);
  smem_attr_once(k_maxvol<T>);
  // algorithmic work: LU pivoting n r^2 plus B = U P^{-1} 2 n r^2
  TT_KERNEL(ex, K_MAXVOL, 3.0 * n * (double)r * r, (8.0 + 2.0 * sizeof(T)) * n * (double)r,
            k_maxvol<T><<<1, MV_THREADS, smem, ex.s>>>(U, n, r, delta, max_iter, W, B, P, I, ex.dev_status));
}

}  // namespace ttfv
