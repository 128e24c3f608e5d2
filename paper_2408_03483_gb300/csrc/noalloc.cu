// tt_round_noalloc: TT rounding for callers that cannot allocate device
// memory (code running where cudaMalloc is unavailable or forbidden, e.g. a
// host that only hands out pre-registered buffers, or a fixed-footprint
// embedding).  Its scratch is a file-scope device array of fixed size that
// every GPU loading this library holds until process exit.
#include <mutex>

#include "tt_common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

// The shared scratch of every tt_round_noalloc call on a device.
static __device__ __align__(256) unsigned char g_round_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  The array's
// name in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
tt_status scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TT_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_round_scratch) != cudaSuccess || p == nullptr) return TT_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return TT_OK;
}

}  // namespace

extern "C" tt_status tt_round_noalloc(const tt2* x, double tol, int32_t rank_cap, tt2* y, double* err_out,
                                      void* stream) {
  if (!x || !y || x->n1 < 1 || x->n2 < 1 || x->rank < 1 || rank_cap < 1) return TT_ERR_ARG;
  const size_t need = tt_round_workspace_size(x->n1, x->n2, x->rank, rank_cap);
  if (need == 0 || need > kNoAllocScratchBytes) return TT_ERR_ARG;
  void* scratch = nullptr;
  const tt_status st = scratch_for_current_device(&scratch);
  if (st != TT_OK) return st;
  return tt_round(x, tol, rank_cap, y, err_out, scratch, kNoAllocScratchBytes, stream);
}
