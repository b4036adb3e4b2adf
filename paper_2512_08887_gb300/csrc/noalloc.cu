// fbst_execute_noalloc: the whole transform with its intermediates in a static device array.
//
// Some callers cannot allocate device memory when they run the transform: a real-time receive
// loop that must never block in the allocator (cudaMalloc can synchronise the device), or a
// process whose device-memory budget is fixed and checked at start-up. This entry point serves
// them: it launches the same three kernels as fbst_execute, but the intermediate arrays
// (yhat [nblk][L][M] and w [nblk][B][L]) live in one file-scope __device__ array of
// kStaticScratchBytes instead of the plan's workspace, and the call makes no allocation of any
// kind. The caller still passes the input and output buffers, and the plan (built once, earlier,
// by fbst_plan) supplies the read-only tables.
//
// Rules of use:
// - The array is a static of this library: every GPU that loads the library holds
//   kStaticScratchBytes (64 MiB) until the process exits, whether or not this entry point is used.
// - A call whose intermediates need more than kStaticScratchBytes is rejected with
//   FBST_ERR_INVALID before anything is launched (split the blocks over several calls).
// - The plan must belong to the current device: the kernels read the plan's tables and write the
//   current device's array, so a plan of another device is rejected with FBST_ERR_INVALID.
// - On its first call on a device (with that device current) the entry point looks up the
//   array's device address with cudaGetSymbolAddress; make that first call before any stream
//   capture. Later calls on that device reuse the address.
// - All calls share the one array, which keeps whatever the last call left in it. Every
//   kernel writes each intermediate entry before it is read, so nothing needs clearing, but calls
//   that overlap on the GPU (different streams, or several host threads) race on the array and
//   must be serialised by the caller.
// - Tensor-core stage-2 variants keep an operand in the plan; they are not offered here
//   (FBST_ERR_UNSUPPORTED).
#include <mutex>

#include "common.cuh"

namespace fbst {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
}  // namespace

// Device address of g_static_scratch on the current device (host code only sees a host-side
// stand-in for the symbol, which must never be passed to a kernel).
static int static_scratch_address(void** out) {
  int dev = -1;
  FBST_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return FBST_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    FBST_CUDA_TRY(cudaGetSymbolAddress(&addr, g_static_scratch));
    if (!addr) return FBST_ERR_CUDA;
    g_scratch_addr[dev] = addr;
  }
  *out = g_scratch_addr[dev];
  return FBST_OK;
}

}  // namespace fbst

using namespace fbst;

extern "C" int fbst_execute_noalloc(fbst_plan_t p, const void* y, void* bhat, int nblk, void* stream) {
  if (!p || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!y || !bhat || (reinterpret_cast<uintptr_t>(y) & 15u) || (reinterpret_cast<uintptr_t>(bhat) & 15u))
    return FBST_ERR_INVALID;
  const fbst_info& in = p->info;
  const size_t yhat_bytes = sizeof(float2) * (size_t)nblk * in.L * in.M;
  const size_t yhat_span = (yhat_bytes + 255) & ~size_t(255);
  const size_t w_bytes = sizeof(float2) * (size_t)nblk * in.B * in.L;
  if (yhat_span + w_bytes > kStaticScratchBytes) {
    set_last_cuda_error(cudaSuccess, "fbst_execute_noalloc: intermediates exceed the 64 MiB static array",
                        __FILE__, __LINE__);
    return FBST_ERR_INVALID;
  }
  if (nblk > 65535) return FBST_ERR_INVALID;
  const int kind = in.stage2;
  if (kind != FBST_STAGE2_GS && kind != FBST_STAGE2_GS_IR1 && kind != FBST_STAGE2_DENSE_FP32)
    return FBST_ERR_UNSUPPORTED;
  int cur = -1;
  FBST_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != p->device) return FBST_ERR_INVALID;
  void* base = nullptr;
  const int st = static_scratch_address(&base);
  if (st != FBST_OK) return st;
  float2* yhat = static_cast<float2*>(base);
  float2* w = reinterpret_cast<float2*>(static_cast<unsigned char*>(base) + yhat_span);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int r = launch_czt_time(p, static_cast<const float2*>(y), yhat, nblk, s);
  if (r == FBST_OK) r = launch_czt_space(p, yhat, w, nblk, s);
  if (r == FBST_OK) {
    r = kind == FBST_STAGE2_DENSE_FP32 ? launch_stage2_dense_fp32(p, w, static_cast<float2*>(bhat), nblk, s)
                                       : launch_stage2_gs(p, w, static_cast<float2*>(bhat), nblk, s);
  }
  return r;
}
