// Dense contractions on the 5th-generation tensor cores (tcgen05) for the
// TF32 and BF16 precision forms: C = alpha A B + beta C with FP32 results.
//
// Operands are first packed K-major (row r of a packed operand holds its K
// entries contiguously) and split into tensor-core parts whose products sum
// to FP32 accuracy: TF32 uses x = hi + lo (3 products: hi*hi + hi*lo +
// lo*hi), BF16 uses x = hi + mid + lo (6 products with weight >= 2^-16).
// The parts are laid side by side along K, so one ordinary K loop over the
// packed operands accumulates every product into the same FP32 accumulator.
//
// Kernel: one CTA per 128 x BN output tile and K slice (split-K for the
// skinny range-finder products).  Warp 0 lane 0 streams 128-byte-wide K
// tiles of A and B into a ring of shared-memory stages by TMA
// (cp.async.bulk.tensor, 128-byte swizzle); warp 1 lane 0 issues
// tcgen05.mma into a TMEM accumulator and releases each stage with
// tcgen05.commit; all four warps then read the accumulator with tcgen05.ld
// (warp w owns TMEM lanes 32w..32w+31 = output rows) and store columns
// coalesced.  Every mbarrier wait is bounded; a timeout latches
// DEV_TC_TIMEOUT in the device status word and the CTA still frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "tt_common.cuh"

namespace ttfv {
namespace {

constexpr int TC_BM = 128;       // output rows per CTA (TMEM lanes)
constexpr int TC_THREADS = 128;  // four warps
constexpr int TC_ROW_BYTES = 128;  // K bytes per stage row (one swizzle span)
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete, at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
// D (TMEM) (+)= A (smem desc) * B (smem desc); KIND 0: tf32, 1: bf16 (kind::f16)
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (KIND == 0)
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte rows in
// the 128-byte swizzle layout TMA writes: 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused: K fits one span)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset between 8-row atoms
  d |= (uint64_t)1 << 46;                           // descriptor version of tcgen05
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}
// Instruction descriptor: FP32 accumulator, A and B K-major of the given
// format (kind::tf32: 2 = TF32; kind::f16: 1 = BF16), N >> 3, M >> 4.
template <int KIND>
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | ((KIND == 0 ? 2u : 1u) << 7) | ((KIND == 0 ? 2u : 1u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

struct TcShape {
  int M, N, BN, kb_total, kb_per, stages;
  uint32_t ncols;
};

// ---------------------------------------------------------------- GEMM kernel
template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, TcShape sh,
              float* __restrict__ C, long ldc, long zstride, float alpha, float beta, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  constexpr int KE = TC_ROW_BYTES / (KIND == 0 ? 4 : 2);  // K elements per stage
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t raw = smem_u32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t a_bytes = TC_BM * TC_ROW_BYTES, b_bytes = (uint32_t)sh.BN * TC_ROW_BYTES;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  const int S = sh.stages;
  const uint32_t bars = base + (uint32_t)S * stage_bytes;  // full[S], empty[S], done, tmem slot
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 8u * (S + s); };
  const uint32_t done = bars + 16u * S;
  const uint32_t slot = done + 8u;
  __shared__ int s_fail;

  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * sh.BN;
  const int kb0 = blockIdx.z * sh.kb_per;
  const int nkb = min(sh.kb_total, kb0 + sh.kb_per) - kb0;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) tmem_alloc(slot, sh.ncols);  // warp-wide, converged
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  uint32_t tmem;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(tmem) : "r"(slot) : "memory");

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    int issued = 0;
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (i >= S && !mbar_wait(empty(s), ((i / S) - 1) & 1)) {
        s_fail = 1;
        break;
      }
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      mbar_expect_tx(full(s), stage_bytes);
      tma_load_2d(sa, &ta, (kb0 + i) * KE, m0, full(s));
      tma_load_2d(sa + a_bytes, &tb, (kb0 + i) * KE, n0, full(s));
      issued = i + 1;
    }
    // the last loads into each stage have landed before the CTA may exit
    for (int i = max(0, issued - S); i < issued; ++i)
      if (!mbar_wait(full(i % S), (i / S) & 1)) s_fail = 1;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = tc_idesc<KIND>(TC_BM, sh.BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % S;
      if (!mbar_wait(full(s), (i / S) & 1)) {
        s_fail = 1;
        break;
      }
      tc_fence_after();
      const uint32_t sa = base + (uint32_t)s * stage_bytes;
      const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + a_bytes);
#pragma unroll
      for (int k = 0; k < TC_ROW_BYTES / 32; ++k)  // 32-byte K slices: +2 in the encoded start address
        tc_mma<KIND>(tmem, ad + 2u * k, bd + 2u * k, idesc, (i > 0 || k > 0) ? 1u : 0u);
      tc_commit(empty(s));
    }
    tc_commit(done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // warp-uniform decision: tcgen05.ld below is a converged warp-wide load
  const bool got = __all_sync(0xffffffffu, mbar_wait(done, 0) ? 1 : 0) != 0;
  tc_fence_after();
  if (!got) s_fail = 1;
  if (got) {
    const int row = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < sh.BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      if (row < sh.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = n0 + c0 + j;
          if (col < sh.N) {
            const float v = __uint_as_float(r[j]);
            if (zstride) {
              C[(size_t)blockIdx.z * zstride + row + (size_t)col * sh.M] = v;
            } else {
              float* c = C + row + (size_t)col * ldc;
              *c = (beta == 0.0f) ? alpha * v : fmaf(alpha, v, beta * *c);
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, sh.ncols);
  if (threadIdx.x == 0 && s_fail) atomicOr(status, (unsigned)DEV_TC_TIMEOUT);
}

// C = alpha * sum_z P[z] + beta * C over the split-K partials (M x N, ld M)
__global__ void k_tc_reduce(int M, int N, int nsplit, const float* __restrict__ P, float alpha, float beta,
                            float* __restrict__ C, long ldc) {
  const long total = (long)M * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int z = 0; z < nsplit; ++z) s += P[t + (size_t)z * total];
    float* c = C + (t % M) + (size_t)(t / M) * ldc;
    *c = (beta == 0.0f) ? alpha * s : fmaf(alpha, s, beta * *c);
  }
}

// ---------------------------------------------------------------- packing
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Packed operand row r (r < rows_p), K' = parts * Kp: dst[r * K' + q * Kp + k]
// = part q of X(r, k) (zero outside rows x K).  TF32 parts (hi, hi, lo) for A
// and (hi, lo, hi) for B; BF16 parts (h, h, m, h, l, m) for A and
// (h, m, h, l, h, m) for B, so that the K' contraction sums the products
// hi*hi + hi*lo + lo*hi (TF32) or hh + hm + mh + hl + lh + mm (BF16).
template <typename Src, int KIND>
__global__ void k_tc_pack(const Src* __restrict__ X, long rs, long cs, int rows, int K, int rows_p, int Kp,
                          int parts, int side, void* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const bool rows_fast = (rs == 1);
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int rr = rows_fast ? r0 + threadIdx.x : r0 + dy;
    const int kk = rows_fast ? k0 + dy : k0 + threadIdx.x;
    const float v = (rr < rows && kk < K) ? (float)X[rr * rs + kk * cs] : 0.0f;
    if (rows_fast)
      tile[threadIdx.x][dy] = v;
    else
      tile[dy][threadIdx.x] = v;
  }
  __syncthreads();
  const long Kq = (long)parts * Kp;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int rr = r0 + dy, kk = k0 + threadIdx.x;
    if (rr >= rows_p || kk >= Kp) continue;
    const float x = tile[dy][threadIdx.x];
    if constexpr (KIND == 0) {
      const float hi = to_tf32(x), lo = to_tf32(x - hi);
      float* d = static_cast<float*>(dst) + (size_t)rr * Kq + kk;
      if (parts == 1) {
        d[0] = hi;
      } else {  // A: hi hi lo ; B: hi lo hi
        d[0] = hi;
        d[Kp] = side == 0 ? hi : lo;
        d[2L * Kp] = side == 0 ? lo : hi;
      }
    } else {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const float r1 = x - __bfloat162float(h);
      const __nv_bfloat16 m = __float2bfloat16_rn(r1);
      const __nv_bfloat16 l = __float2bfloat16_rn(r1 - __bfloat162float(m));
      __nv_bfloat16* d = static_cast<__nv_bfloat16*>(dst) + (size_t)rr * Kq + kk;
      if (parts == 1) {
        d[0] = h;
      } else {  // A: h h m h l m ; B: h m h l h m
        const __nv_bfloat16 a[6] = {h, h, m, h, l, m};
        const __nv_bfloat16 b[6] = {h, m, h, l, h, m};
#pragma unroll
        for (int q = 0; q < 6; ++q) d[(long)q * Kp] = side == 0 ? a[q] : b[q];
      }
    }
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2-D map over a packed operand (rows x kq elements, row-major), box of
// box_rows x 128 bytes with the 128-byte swizzle
CUtensorMap make_map(const void* base, int kind, long rows, long kq, int box_rows) {
  auto enc = tensor_map_encoder();
  TT_REQUIRE(enc != nullptr, TT_ERR_CUDA);
  const int esize = kind == 0 ? 4 : 2;
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  const cuuint64_t dims[2] = {(cuuint64_t)kq, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kq * esize};
  const cuuint32_t box[2] = {(cuuint32_t)(TC_ROW_BYTES / esize), (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&m, kind == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  TT_REQUIRE(r == CUDA_SUCCESS, TT_ERR_CUDA);
  return m;
}

int grid_1d(long n) { return std::max(1, std::min(ceil_div(n, 256), 1184)); }

template <typename Src>
void pack(Exec& ex, int kind, const Src* X, long rs, long cs, int rows, int K, int rows_p, int Kp, int parts,
          int side, void* dst) {
  dim3 grid(ceil_div(Kp, 32), ceil_div(rows_p, 32));
  const double bytes = (double)sizeof(Src) * rows * K + (kind == 0 ? 4.0 : 2.0) * parts * (double)rows_p * Kp;
  if (kind == 0)
    TT_KERNEL(ex, K_OTHER, 0, bytes,
              (k_tc_pack<Src, 0><<<grid, dim3(32, 8), 0, ex.s>>>(X, rs, cs, rows, K, rows_p, Kp, parts, side,
                                                                  dst)));
  else
    TT_KERNEL(ex, K_OTHER, 0, bytes,
              (k_tc_pack<Src, 1><<<grid, dim3(32, 8), 0, ex.s>>>(X, rs, cs, rows, K, rows_p, Kp, parts, side,
                                                                  dst)));
}

}  // namespace

int tc_parts(int precision, bool split) {
  if (!split) return 1;
  return precision == TT_BF16 ? 6 : 3;
}

// C (M x N, col-major ld ldc, FP32) = alpha A B + beta C on tcgen05;
// A(i, k) = A[i*ars + k*acs], B(k, j) = B[k*brs + j*bcs].
template <typename Src>
void tc_gemm(Exec& ex, int precision, bool split, int M, int N, int K, float alpha, const Src* A, long ars,
             long acs, const Src* B, long brs, long bcs, float beta, float* C, long ldc) {
  TT_REQUIRE(precision == TT_TF32 || precision == TT_BF16, TT_ERR_ARG);
  if (M <= 0 || N <= 0) return;
  TT_REQUIRE(K >= 1, TT_ERR_ARG);
  const int kind = precision == TT_TF32 ? 0 : 1;
  const int esize = kind == 0 ? 4 : 2;
  const int KE = TC_ROW_BYTES / esize;
  const int parts = tc_parts(precision, split);
  const int Kp = ceil_div(K, KE) * KE;
  const int Mp = ceil_div(M, TC_BM) * TC_BM;
  const int BN = N <= 256 ? ceil_div(N, 16) * 16 : 128;
  const int nt = ceil_div(N, BN);
  const int Np = nt * BN;
  const int mt = Mp / TC_BM;
  TcShape sh;
  sh.M = M;
  sh.N = N;
  sh.BN = BN;
  sh.kb_total = parts * Kp / KE;
  // split K so that the grid covers the SMs about once
  int nsplit = std::max(1, std::min(sh.kb_total, sm_count() / std::max(1, mt * nt)));
  sh.kb_per = ceil_div(sh.kb_total, nsplit);
  nsplit = ceil_div(sh.kb_total, sh.kb_per);
  const uint32_t stage_bytes = (uint32_t)(TC_BM + BN) * TC_ROW_BYTES;
  sh.stages = std::max(2, std::min(6, (int)((200u * 1024u) / stage_bytes)));
  uint32_t nc = 32;
  while (nc < (uint32_t)BN) nc <<= 1;
  sh.ncols = nc;
  Scope sc(*ex.ar);
  void* Ap = ex.ar->get<unsigned char>((size_t)Mp * parts * Kp * esize);
  void* Bp = ex.ar->get<unsigned char>((size_t)Np * parts * Kp * esize);
  float* P = nsplit > 1 ? ex.ar->get<float>((size_t)nsplit * M * N) : nullptr;
  if (ex.dry) return;
  pack(ex, kind, A, ars, acs, M, K, Mp, Kp, parts, 0, Ap);
  // B^T (N x K): row j, entry k = B(k, j)
  pack(ex, kind, B, bcs, brs, N, K, Np, Kp, parts, 1, Bp);
  const CUtensorMap ma = make_map(Ap, kind, Mp, (long)parts * Kp, TC_BM);
  const CUtensorMap mb = make_map(Bp, kind, Np, (long)parts * Kp, BN);
  const size_t smem = 1024 + (size_t)sh.stages * stage_bytes + 8 * (2 * sh.stages + 2) + 64;
  dim3 grid(mt, nt, nsplit);
  const double fl = 2.0 * M * (double)N * K * parts;
  const double by = (double)esize * parts * Kp * ((double)Mp * nt + (double)Np * mt) + 4.0 * M * (double)N * nsplit;
  float* out = nsplit > 1 ? P : C;
  const long zs = nsplit > 1 ? (long)M * N : 0;
  if (kind == 0) {
    smem_attr_once(k_tc_gemm<0>);
    TT_KERNEL(ex, K_GEMM, fl, by,
              (k_tc_gemm<0><<<grid, TC_THREADS, smem, ex.s>>>(ma, mb, sh, out, ldc, zs, alpha, beta,
                                                               ex.dev_status)));
  } else {
    smem_attr_once(k_tc_gemm<1>);
    TT_KERNEL(ex, K_GEMM, fl, by,
              (k_tc_gemm<1><<<grid, TC_THREADS, smem, ex.s>>>(ma, mb, sh, out, ldc, zs, alpha, beta,
                                                               ex.dev_status)));
  }
  if (nsplit > 1) {
    const long total = (long)M * N;
    TT_KERNEL(ex, K_GEMM, (double)nsplit * total, 4.0 * total * (nsplit + (beta == 0.0f ? 1 : 2)),
              k_tc_reduce<<<grid_1d(total), 256, 0, ex.s>>>(M, N, nsplit, P, alpha, beta, C, ldc));
  }
}

template void tc_gemm<float>(Exec&, int, bool, int, int, int, float, const float*, long, long, const float*, long,
                             long, float, float*, long);
template void tc_gemm<double>(Exec&, int, bool, int, int, int, float, const double*, long, long, const double*,
                              long, long, float, float*, long);

}  // namespace ttfv
