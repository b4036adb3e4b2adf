// Calibration: the FP32 CUDA-core throughput of the current device, measured, as the denominator
// of the ALU roofline of the FFT kernels. No counterpart in the paper.
//
// Every thread runs kChains independent FMA chains (a = a * m + c, so every instruction is one
// FFMA = 2 flops with no dependence between chains within an iteration); the grid is the resident
// CTAs of the device (8 CTAs of 256 threads per SM), so every FP32 lane is busy and the dependent
// latency of one chain is hidden by the other chains and warps. The result is stored only if it
// equals a value it cannot reach (so the compiler must keep every FMA), and the time is taken with
// CUDA events on the caller's stream.
#include "common.cuh"
#include "launch_util.cuh"

namespace fbst {

constexpr int kChains = 8;
constexpr int kFmaThreads = 256;

__global__ void __launch_bounds__(kFmaThreads) k_fma_chain(float* sink, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == -1.2345678e30f) sink[0] = s;
}

}  // namespace fbst

using namespace fbst;

extern "C" int fbst_fp32_fma_peak(void* sink, int iters, double* tflops, double* ms, void* stream) {
  if (!sink || !tflops || iters <= 0 || (reinterpret_cast<uintptr_t>(sink) & 3u)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int grid = sm_count() * 8;
  // m slightly below 1 and c small keep every chain finite for any iteration count.
  const float m = 0.999999f, c = 1e-7f;
  cudaEvent_t e0, e1;
  FBST_CUDA_TRY(cudaEventCreate(&e0));
  FBST_CUDA_TRY(cudaEventCreate(&e1));
  k_fma_chain<<<grid, kFmaThreads, 0, s>>>(static_cast<float*>(sink), iters, m, c);  // warm-up
  cudaEventRecord(e0, s);
  k_fma_chain<<<grid, kFmaThreads, 0, s>>>(static_cast<float*>(sink), iters, m, c);
  cudaEventRecord(e1, s);
  const cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  if (err == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  FBST_CUDA_TRY(err);
  FBST_CUDA_TRY(cudaGetLastError());
  const double flops = 2.0 * kChains * 16.0 * (double)iters * (double)grid * kFmaThreads;
  *tflops = t > 0.f ? flops / (t * 1e-3) / 1e12 : 0.0;
  if (ms) *ms = t;
  return FBST_OK;
}
