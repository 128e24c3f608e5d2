// Learned-pivot network: a 3-layer perceptron (14 -> 256 -> 256 -> 1) that
// scores the column indices of a cross from features of the cross's initial
// TT and of the call site's previous pivots; its top-scoring indices seed the
// maxvol sweeps.  Training products (forward and backward) run on the
// tcgen05 tensor cores with BF16 operands and FP32 accumulation (tc_gemm, one
// part); scoring for a cross uses one fused CUDA-core kernel with the same
// BF16-operand products; biases, activations, the logistic loss and the Adam
// update are FP32 elementwise kernels.
//
// Layouts: activations and features are column-major m x width (ld m);
// W1 (12 x 256) and W2 (256 x 256) are row-major (W[in * 256 + out]).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tt_ops.cuh"

namespace ttfv {

constexpr int MLP_F = 14;
constexpr int MLP_H = 256;

namespace {

int grid_for(long n) { return std::max(1, std::min(ceil_div(n, 256), 1184)); }

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void k_bias_relu(float* __restrict__ Z, float* __restrict__ H, int m, int n,
                            const float* __restrict__ b) {
  const long total = (long)m * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const float z = Z[t] + b[t / m];
    Z[t] = z;
    H[t] = z > 0.0f ? z : 0.0f;
  }
}
__global__ void k_add_scalar(float* __restrict__ s, int m, const float* __restrict__ b) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) s[t] += b[0];
}
// ds = (sigmoid(s) - y) / m; per-block partial sums of the logistic loss
__global__ void k_loss_ds(const float* __restrict__ s, const float* __restrict__ y, int m, float* __restrict__ ds,
                          double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m; t += gridDim.x * blockDim.x) {
    const double sv = s[t], yv = y[t];
    acc += fmax(sv, 0.0) + log1p(exp(-fabs(sv))) - yv * sv;
    ds[t] = (float)((1.0 / (1.0 + exp(-sv)) - yv) / m);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
__global__ void k_sum_blocks(const double* __restrict__ part, int n, int m, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += part[i];
    *out = t / m;
  }
}
// dZ2 = (bf16(ds) outer bf16(w3)) masked by Z2 > 0
__global__ void k_dz2(const float* __restrict__ ds, const float* __restrict__ w3, const float* __restrict__ Z2, int m,
                      float* __restrict__ dZ2) {
  const long total = (long)m * MLP_H;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t % m), h = (int)(t / m);
    dZ2[t] = Z2[t] > 0.0f ? bf16r(ds[i]) * bf16r(w3[h]) : 0.0f;
  }
}
__global__ void k_mask(float* __restrict__ dH, const float* __restrict__ Z, long total) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x)
    if (!(Z[t] > 0.0f)) dH[t] = 0.0f;
}
// g[j] = sum_i D[i + j m] (one block per column, FP64 accumulation)
__global__ void k_colsum(const float* __restrict__ D, int m, float* __restrict__ g) {
  __shared__ double red[32];
  const float* d = D + (size_t)blockIdx.x * m;
  double acc = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) acc += d[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g[blockIdx.x] = (float)t;
  }
}
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float c1, float c2) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const float gv = g[t];
    const float a = 0.9f * m1[t] + 0.1f * gv;
    const float b = 0.999f * m2[t] + 0.001f * gv * gv;
    m1[t] = a;
    m2[t] = b;
    p[t] -= lr * (a / c1) / (sqrtf(b / c2) + 1e-8f);
  }
}

// ---- features of the column mode of x0 = A B^T
// raw per-index values: leverage of the orthonormal basis Q of B, column
// mean c_j = B[j,:] . mean(A), energy e_j = B[j,:] G B[j,:]^T (BG = B G given)
__global__ void k_feat_raw(const double* __restrict__ Q, const double* __restrict__ B, const double* __restrict__ BG,
                           const double* __restrict__ amean, int n2, int r, double* __restrict__ raw) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
    double l = 0.0, c = 0.0, e = 0.0;
    for (int k = 0; k < r; ++k) {
      const double q = Q[j + (size_t)k * n2], b = B[j + (size_t)k * n2];
      l = fma(q, q, l);
      c = fma(b, amean[k], c);
      e = fma(b, BG[j + (size_t)k * n2], e);
    }
    raw[j] = l * ((double)n2 / r);
    raw[n2 + j] = c;
    raw[2 * n2 + j] = e;
  }
}
// stats: mean c, std c (population), mean |d2|, mean e -> st[0..3]; one CTA
__global__ void k_feat_stats(const double* __restrict__ raw, int n2, double* __restrict__ st) {
  __shared__ double red[4][32];
  const double* c = raw + n2;
  const double* e = raw + 2 * n2;
  double sc = 0.0, sd2 = 0.0, se = 0.0, sa = 0.0;
  for (int j = threadIdx.x; j < n2; j += blockDim.x) {
    const double cj = c[j];
    const double d2 = c[(j + 1) % n2] - 2.0 * cj + c[(j + n2 - 1) % n2];
    sc += cj;
    sa += fabs(cj);
    sd2 += fabs(d2);
    se += e[j];
  }
  for (int o = 16; o > 0; o >>= 1) {
    sc += __shfl_xor_sync(0xffffffffu, sc, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sd2 += __shfl_xor_sync(0xffffffffu, sd2, o);
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][w] = sc;
    red[1][w] = sa;
    red[2][w] = sd2;
    red[3][w] = se;
  }
  __syncthreads();
  __shared__ double mean_c;
  if (threadIdx.x == 0) {
    double a = 0, b = 0, d = 0, f = 0;
    for (int i = 0; i < nw; ++i) {
      a += red[0][i];
      b += red[1][i];
      d += red[2][i];
      f += red[3][i];
    }
    mean_c = a / n2;
    st[0] = a / n2;
    st[4] = b / n2;  // mean |c|
    st[2] = d / n2;
    st[3] = f / n2;
  }
  __syncthreads();
  double v = 0.0;
  for (int j = threadIdx.x; j < n2; j += blockDim.x) {
    const double dc = c[j] - mean_c;
    v = fma(dc, dc, v);
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[0][w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < nw; ++i) a += red[0][i];
    st[1] = sqrt(a / n2);
  }
}
__global__ void k_feat_fill(const double* __restrict__ raw, const double* __restrict__ st, int n2,
                            const int* __restrict__ prev, int nprev, float* __restrict__ X) {
  const double* lev = raw;
  const double* c = raw + n2;
  const double* e = raw + 2 * n2;
  const double sdr = st[1];
  const double sd = sdr > 1e-12 * st[4] ? sdr : 1.0;
  const double me = st[3] > 0.0 ? st[3] : 1.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n2; j += gridDim.x * blockDim.x) {
    const int jp = (j + 1) % n2, jm = (j + n2 - 1) % n2;
    const double d2 = c[jp] - 2.0 * c[j] + c[jm];
    const double ang = 2.0 * 3.14159265358979323846 * (double)j / n2;
    double f[MLP_F];
    f[0] = lev[j];
    f[1] = lev[(j + n2 - 2) % n2];
    f[2] = lev[jm];
    f[3] = lev[jp];
    f[4] = lev[(j + 2) % n2];
    f[5] = (c[j] - st[0]) / sd;
    f[6] = 0.5 * (c[jp] - c[jm]) / sd;
    f[7] = d2 / sd;
    f[8] = log1p(fabs(d2) / (st[2] + 1e-300));
    f[9] = e[j] / me;
    f[10] = sin(ang);
    f[11] = cos(ang);
    // previous converged pivots of the same cross site: indicator and
    // periodic distance, capped at 8 (1 when there are none)
    int dmin = 8;
    for (int q = 0; q < nprev; ++q) {
      int dd = abs(j - prev[q]);
      dd = min(dd, n2 - dd);
      dmin = min(dmin, dd);
    }
    f[12] = (nprev > 0 && dmin == 0) ? 1.0 : 0.0;
    f[13] = dmin / 8.0;
#pragma unroll
    for (int q = 0; q < MLP_F; ++q) X[j + (size_t)q * n2] = (float)f[q];
  }
}
__global__ void k_colmean(const double* __restrict__ A, int n1, int r, double* __restrict__ out) {
  __shared__ double red[32];
  const double* a = A + (size_t)blockIdx.x * n1;
  double s = 0.0;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) s += a[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[blockIdx.x] = t / n1;
  }
}

// k highest scores (ties to the smaller index), returned ascending; one CTA
__global__ void __launch_bounds__(1024) k_topk(const float* __restrict__ s, int m, int k, float* __restrict__ work,
                                               int* __restrict__ idx) {
  __shared__ float bv[32];
  __shared__ int bi[32];
  __shared__ int sel[128];
  for (int t = threadIdx.x; t < m; t += blockDim.x) work[t] = s[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < k; ++q) {
    float v = -INFINITY;
    int id = 0x7fffffff;
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
      const float x = work[t];
      if (x > v || (x == v && t < id)) {
        v = x;
        id = t;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, id, o);
      if (v2 > v || (v2 == v && i2 < id)) {
        v = v2;
        id = i2;
      }
    }
    if (lane == 0) {
      bv[w] = v;
      bi[w] = id;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float bvv = bv[0];
      int bii = bi[0];
      for (int u = 1; u < nw; ++u)
        if (bv[u] > bvv || (bv[u] == bvv && bi[u] < bii)) {
          bvv = bv[u];
          bii = bi[u];
        }
      if (bii < 0 || bii >= m) bii = 0;  // all -inf: cannot happen for k <= m
      sel[q] = bii;
      work[bii] = -INFINITY;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int a = 1; a < k; ++a) {  // insertion sort, k <= 128
      const int x = sel[a];
      int b = a - 1;
      while (b >= 0 && sel[b] > x) {
        sel[b + 1] = sel[b];
        --b;
      }
      sel[b + 1] = x;
    }
    for (int a = 0; a < k; ++a) idx[a] = sel[a];
  }
}

// Fused scoring of a tile of 32 rows per CTA, one thread per hidden unit:
// the same products as the tensor-core passes (operands rounded to BF16,
// FP32 accumulation), with both hidden layers kept in shared memory -- the
// cross's proposals score a few hundred to a few thousand rows, where one
// launch beats a chain of GEMM launches.
constexpr int INF_ROWS = 32;
__global__ void __launch_bounds__(MLP_H) k_mlp_infer(const float* __restrict__ X, int m,
                                                     const float* __restrict__ W1, const float* __restrict__ b1,
                                                     const float* __restrict__ W2, const float* __restrict__ b2,
                                                     const float* __restrict__ w3, const float* __restrict__ b3,
                                                     float* __restrict__ s) {
  __shared__ float xs[INF_ROWS][MLP_F];
  __shared__ float hs[INF_ROWS][MLP_H + 1];
  const int h = threadIdx.x, r0 = blockIdx.x * INF_ROWS;
  const int nr = min(INF_ROWS, m - r0);
  for (int t = threadIdx.x; t < INF_ROWS * MLP_F; t += blockDim.x) {
    const int r = t % INF_ROWS, f = t / INF_ROWS;
    xs[r][f] = r < nr ? bf16r(X[(r0 + r) + (size_t)f * m]) : 0.0f;
  }
  __syncthreads();
  // layer 1: unit h over the tile's rows
  float w1[MLP_F];
#pragma unroll
  for (int f = 0; f < MLP_F; ++f) w1[f] = bf16r(W1[f * MLP_H + h]);
  const float bb1 = b1[h];
  for (int r = 0; r < INF_ROWS; ++r) {
    float z = 0.0f;
#pragma unroll
    for (int f = 0; f < MLP_F; ++f) z = fmaf(xs[r][f], w1[f], z);
    z += bb1;
    hs[r][h] = bf16r(z > 0.0f ? z : 0.0f);
  }
  __syncthreads();
  // layer 2: unit h of the second layer, W2 column h streamed from L2
  float acc[INF_ROWS];
#pragma unroll
  for (int r = 0; r < INF_ROWS; ++r) acc[r] = 0.0f;
  for (int k = 0; k < MLP_H; ++k) {
    const float w = bf16r(W2[(size_t)k * MLP_H + h]);
#pragma unroll
    for (int r = 0; r < INF_ROWS; ++r) acc[r] = fmaf(hs[r][k], w, acc[r]);
  }
  __syncthreads();
  // layer 3: per-row dot with w3 through shared memory
  const float ww3 = bf16r(w3[h]), bb2 = b2[h];
#pragma unroll
  for (int r = 0; r < INF_ROWS; ++r) {
    const float z = acc[r] + bb2;
    hs[r][h] = bf16r(z > 0.0f ? z : 0.0f) * ww3;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (int r = wp; r < nr; r += MLP_H / 32) {
    float v = 0.0f;
    for (int k = lane; k < MLP_H; k += 32) v += hs[r][k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s[r0 + r] = v + b3[0];
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
void mlp_features(Exec& ex, const TT& x0, const int* prev, int nprev, float* X) {
  const int n1 = x0.n1, n2 = x0.n2, r = x0.r;
  TT_REQUIRE(r >= 1 && r <= 112 && n2 >= 1, TT_ERR_ARG);
  Scope sc(*ex.ar);
  QRTree tb;
  tsqr(ex, x0.b, n2, r, n2, tb);
  double* Iden = ex.ar->get<double>((size_t)r * r);
  double* Q = ex.ar->get<double>((size_t)n2 * r);
  set_identity(ex, Iden, r);
  tsqr_apply(ex, tb, Iden, r, r, Q, n2);
  double* G = ex.ar->get<double>((size_t)r * r);
  double* BG = ex.ar->get<double>((size_t)n2 * r);
  double* amean = ex.ar->get<double>(r);
  double* raw = ex.ar->get<double>((size_t)3 * n2);
  double* st = ex.ar->get<double>(8);
  gemm<double>(ex, r, r, n1, 1.0, x0.a, n1, 1, x0.a, 1, n1, 0.0, G, r);  // A^T A
  gemm<double>(ex, n2, r, r, 1.0, x0.b, 1, n2, G, 1, r, 0.0, BG, n2);    // B G
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, 0, 8.0 * n1 * r, k_colmean<<<r, 256, 0, ex.s>>>(x0.a, n1, r, amean));
  TT_KERNEL(ex, K_OTHER, 6.0 * n2 * r, 8.0 * (3.0 * n2 * r + 3.0 * n2),
            k_feat_raw<<<grid_for(n2), 256, 0, ex.s>>>(Q, x0.b, BG, amean, n2, r, raw));
  TT_KERNEL(ex, K_OTHER, 8.0 * n2, 16.0 * n2, k_feat_stats<<<1, 1024, 0, ex.s>>>(raw, n2, st));
  TT_KERNEL(ex, K_OTHER, 20.0 * n2 + 3.0 * n2 * nprev, 24.0 * n2 + 56.0 * n2,
            k_feat_fill<<<grid_for(n2), 256, 0, ex.s>>>(raw, st, n2, prev, nprev, X));
}

// Cached activations of a forward pass over m rows
struct MlpActs {
  float *Z1, *H1, *Z2, *H2, *s;
};

static MlpActs mlp_forward_acts(Exec& ex, const MlpNet& net, const float* X, int m) {
  MlpActs a;
  a.Z1 = ex.ar->get<float>((size_t)m * MLP_H);
  a.H1 = ex.ar->get<float>((size_t)m * MLP_H);
  a.Z2 = ex.ar->get<float>((size_t)m * MLP_H);
  a.H2 = ex.ar->get<float>((size_t)m * MLP_H);
  a.s = ex.ar->get<float>((size_t)m);
  const long mh = (long)m * MLP_H;
  // Z1 = X W1 (m x 12 col-major, W1 row-major 12 x 256)
  tc_gemm<float>(ex, TT_BF16, false, m, MLP_H, MLP_F, 1.0f, X, 1, m, net.W1, MLP_H, 1, 0.0f, a.Z1, m);
  if (!ex.dry)
    TT_KERNEL(ex, K_OTHER, mh, 12.0 * mh, k_bias_relu<<<grid_for(mh), 256, 0, ex.s>>>(a.Z1, a.H1, m, MLP_H, net.b1));
  tc_gemm<float>(ex, TT_BF16, false, m, MLP_H, MLP_H, 1.0f, a.H1, 1, m, net.W2, MLP_H, 1, 0.0f, a.Z2, m);
  if (!ex.dry)
    TT_KERNEL(ex, K_OTHER, mh, 12.0 * mh, k_bias_relu<<<grid_for(mh), 256, 0, ex.s>>>(a.Z2, a.H2, m, MLP_H, net.b2));
  tc_gemm<float>(ex, TT_BF16, false, m, 1, MLP_H, 1.0f, a.H2, 1, m, net.w3, 1, 1, 0.0f, a.s, m);
  if (!ex.dry) TT_KERNEL(ex, K_OTHER, m, 8.0 * m, k_add_scalar<<<grid_for(m), 256, 0, ex.s>>>(a.s, m, net.b3));
  return a;
}

void mlp_forward(Exec& ex, const MlpNet& net, const float* X, int m, float* s) {
  if (ex.dry || m <= 0) return;
  TT_KERNEL(ex, K_OTHER, 2.0 * m * (double)MLP_H * (MLP_F + MLP_H + 1),
            4.0 * ((double)m * (MLP_F + 1) + ceil_div(m, INF_ROWS) * (double)MLP_H * (MLP_F + MLP_H + 3)),
            k_mlp_infer<<<ceil_div(m, INF_ROWS), MLP_H, 0, ex.s>>>(X, m, net.W1, net.b1, net.W2, net.b2, net.w3,
                                                                    net.b3, s));
}

void mlp_grad(Exec& ex, const MlpNet& net, const float* X, const float* y, int m, const MlpNet& g,
              double* loss) {
  Scope sc(*ex.ar);
  MlpActs a = mlp_forward_acts(ex, net, X, m);
  const long mh = (long)m * MLP_H;
  float* ds = ex.ar->get<float>((size_t)m);
  float* dZ2 = ex.ar->get<float>((size_t)mh);
  float* dZ1 = ex.ar->get<float>((size_t)mh);
  const int lb = std::max(1, std::min(ceil_div(m, 256), 256));
  double* part = ex.ar->get<double>((size_t)lb);
  double* lossbuf = ex.ar->get<double>(1);
  if (!ex.dry) {
    TT_KERNEL(ex, K_OTHER, 8.0 * m, 12.0 * m, k_loss_ds<<<lb, 256, 0, ex.s>>>(a.s, y, m, ds, part));
    TT_KERNEL(ex, K_OTHER, lb, 8.0 * lb, k_sum_blocks<<<1, 32, 0, ex.s>>>(part, lb, m, loss ? loss : lossbuf));
  }
  // g_w3 = H2^T ds ; g_b3 = sum ds
  tc_gemm<float>(ex, TT_BF16, false, MLP_H, 1, m, 1.0f, a.H2, m, 1, ds, 1, m, 0.0f, g.w3, MLP_H);
  if (!ex.dry) {
    TT_KERNEL(ex, K_OTHER, m, 4.0 * m, k_colsum<<<1, 256, 0, ex.s>>>(ds, m, g.b3));
    TT_KERNEL(ex, K_OTHER, mh, 12.0 * mh, k_dz2<<<grid_for(mh), 256, 0, ex.s>>>(ds, net.w3, a.Z2, m, dZ2));
  }
  // g_W2 (row-major h x h') = its transpose col-major: dZ2^T H1 (h' x h)
  tc_gemm<float>(ex, TT_BF16, false, MLP_H, MLP_H, m, 1.0f, dZ2, m, 1, a.H1, 1, m, 0.0f, g.W2, MLP_H);
  if (!ex.dry) TT_KERNEL(ex, K_OTHER, mh, 4.0 * mh, k_colsum<<<MLP_H, 256, 0, ex.s>>>(dZ2, m, g.b2));
  // dH1 = dZ2 W2^T, then the ReLU mask of Z1
  tc_gemm<float>(ex, TT_BF16, false, m, MLP_H, MLP_H, 1.0f, dZ2, 1, m, net.W2, 1, MLP_H, 0.0f, dZ1, m);
  if (!ex.dry) {
    TT_KERNEL(ex, K_OTHER, 0, 12.0 * mh, k_mask<<<grid_for(mh), 256, 0, ex.s>>>(dZ1, a.Z1, mh));
    TT_KERNEL(ex, K_OTHER, mh, 4.0 * mh, k_colsum<<<MLP_H, 256, 0, ex.s>>>(dZ1, m, g.b1));
  }
  // g_W1 (row-major f x h) = its transpose col-major: dZ1^T X (h x f)
  tc_gemm<float>(ex, TT_BF16, false, MLP_H, MLP_F, m, 1.0f, dZ1, m, 1, X, 1, m, 0.0f, g.W1, MLP_H);
}

void mlp_adam(Exec& ex, const MlpNet& p, const MlpNet& g, const MlpNet& m1, const MlpNet& m2, int t, float lr) {
  if (ex.dry) return;
  const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
  float* P[6] = {p.W1, p.b1, p.W2, p.b2, p.w3, p.b3};
  float* G[6] = {g.W1, g.b1, g.W2, g.b2, g.w3, g.b3};
  float* M1[6] = {m1.W1, m1.b1, m1.W2, m1.b2, m1.w3, m1.b3};
  float* M2[6] = {m2.W1, m2.b1, m2.W2, m2.b2, m2.w3, m2.b3};
  const int n[6] = {MLP_F * MLP_H, MLP_H, MLP_H * MLP_H, MLP_H, MLP_H, 1};
  for (int q = 0; q < 6; ++q)
    TT_KERNEL(ex, K_OTHER, 10.0 * n[q], 20.0 * n[q],
              k_adam<<<grid_for(n[q]), 256, 0, ex.s>>>(P[q], G[q], M1[q], M2[q], n[q], lr, c1, c2));
}

void mlp_topk(Exec& ex, const float* s, int m, int k, int* idx) {
  TT_REQUIRE(k >= 1 && k <= 128 && k <= m, TT_ERR_ARG);
  Scope sc(*ex.ar);
  float* work = ex.ar->get<float>((size_t)m);
  if (ex.dry) return;
  TT_KERNEL(ex, K_OTHER, (double)m * k, 8.0 * m, k_topk<<<1, 1024, 0, ex.s>>>(s, m, k, work, idx));
}

// Previous pivots (host) copied to a device array of the arena
static const int* upload_prev(Exec& ex, const std::vector<int>& prev) {
  int* d = ex.ar->get<int>(std::max<size_t>(prev.size(), 1));
  if (!ex.dry && !prev.empty())
    TT_CUDA(cudaMemcpyAsync(d, prev.data(), sizeof(int) * prev.size(), cudaMemcpyHostToDevice, ex.s));
  return d;
}

void mlp_features_host_prev(Exec& ex, const TT& x0, const std::vector<int>& prev, float* X) {
  Scope sc(*ex.ar);
  const int* dprev = upload_prev(ex, prev);
  mlp_features(ex, x0, dprev, (int)prev.size(), X);
}

// Column pivots proposed by the network for a cross whose initial TT is x0
void mlp_propose(Exec& ex, const MlpNet& net, const TT& x0, const std::vector<int>& prev, int k, int* idx) {
  Scope sc(*ex.ar);
  float* X = ex.ar->get<float>((size_t)x0.n2 * MLP_F);
  float* s = ex.ar->get<float>((size_t)x0.n2);
  mlp_features_host_prev(ex, x0, prev, X);
  mlp_forward(ex, net, X, x0.n2, s);
  mlp_topk(ex, s, x0.n2, k, idx);
}

}  // namespace ttfv
