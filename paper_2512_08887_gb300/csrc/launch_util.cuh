// Launch helpers shared by the stage kernels: work ranges and grids sized to the resident CTAs.
#pragma once

#include <algorithm>
#include <mutex>
#include <unordered_set>

#include "common.cuh"

namespace fbst {

constexpr size_t kMaxSmem = 227 * 1024;

#ifndef FBST_TRY
#define FBST_TRY(expr)                      \
  do {                                      \
    const int fbst_r_ = (expr);             \
    if (fbst_r_ != FBST_OK) return fbst_r_; \
  } while (0)
#endif

// CTA blockIdx.x of gridDim.x takes the contiguous range [c*I/G, (c+1)*I/G) of I work items.
__device__ __forceinline__ void my_range(long long items, long long* begin, long long* end) {
  const long long G = gridDim.x, c = blockIdx.x;
  *begin = items * c / G;
  *end = items * (c + 1) / G;
}

inline int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  return sms;
}

// Resident CTAs of `kernel` on the current device for the given block size and shared memory.
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return sm_count() * per_sm;
}

inline int grid_for_items(long long items, int slots) {
  return (int)std::max<long long>(1, std::min<long long>(items, slots));
}

// Allow the kernel the full 227 KB of dynamic shared memory (once per kernel).
template <typename K>
int allow_max_smem(K kernel) {
  static std::mutex mu;
  static std::unordered_set<const void*> done;
  std::lock_guard<std::mutex> lock(mu);
  const void* key = reinterpret_cast<const void*>(kernel);
  if (!done.count(key)) {
    FBST_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem));
    done.insert(key);
  }
  return FBST_OK;
}

}  // namespace fbst
