// Streaming over contiguous, overlapping blocks (Sec. III-A: the batches of snapshots may be
// contiguous and overlap).
//
// A continuous record [M][T] (sample fastest) is cut into blocks of N snapshots starting every `hop`
// samples; stage 1a reads each block in place from the record (no copy), stages 1b and 2 run as for
// fbst_execute, and every block contributes its central `hop` output samples, [c, c + hop) with
// c = (N - hop)/2, to one continuous output stream per beam: stream sample k*hop + i is output
// sample c + i of block k, the beam at record time c + k*hop + i. Dropping the samples near the
// block edges, where the Fourier extension of a block fits worst, lowers the bias of the stream
// below that of non-overlapping blocks.
#include <algorithm>

#include "common.cuh"
#include "launch_util.cuh"

namespace fbst {
namespace {

// out[b][(k0 + k)*hop + i] = bhat[k][b][c + i] for k < nb, i < hop (one thread per output value).
__global__ void k_stream_emit(const float2* __restrict__ bhat, float2* __restrict__ out, int B, int N, int hop, int c,
                              long long out_len, int k0, int nb) {
  const long long total = (long long)nb * B * hop;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e % hop);
    const long long kb = e / hop;
    const int b = (int)(kb % B), k = (int)(kb / B);
    out[(size_t)b * out_len + (size_t)(k0 + k) * hop + i] = bhat[((size_t)k * B + b) * N + c + i];
  }
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

}  // namespace
}  // namespace fbst

using namespace fbst;

extern "C" int fbst_execute_stream(fbst_plan_t p, const void* record, long long T, int hop, void* out, int nblk,
                                   void* stream) {
  if (!p || nblk < 0 || T < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  const fbst_info& in = p->info;
  if (!record || !out || !aligned16(record) || !aligned16(out)) return FBST_ERR_INVALID;
  if (hop < 1 || hop > in.N || (in.N - hop) % 2 != 0) return FBST_ERR_INVALID;
  if ((long long)(nblk - 1) * hop + in.N > T) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int maxb = std::min(p->band.max_blocks, 65535);
  // The blocks' outputs before their central parts are emitted: plan memory, allocated on first
  // use through the plan's allocator (like the host path's staging).
  if (!p->stream_bhat) {
    FBST_TRY(plan_alloc_n(p, &p->stream_bhat, (size_t)maxb * in.B * in.N));
    FBST_CUDA_TRY(cudaStreamSynchronize(p->mem_stream));
  }
  const int c = (in.N - hop) / 2;
  const long long out_len = (long long)nblk * hop;
  const float2* rec = static_cast<const float2*>(record);
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(launch_czt_time_record(p, rec + (size_t)c0 * hop, T, hop, p->ws_yhat, nb, s));
    FBST_TRY(launch_czt_space_scaled(p, p->ws_yhat, p->ws_w, nb, 0, s));
    FBST_TRY(run_stage2(p, p->ws_w, p->stream_bhat, nb, s, true));
    const long long total = (long long)nb * in.B * hop;
    const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, (long long)sm_count() * 8));
    k_stream_emit<<<grid, 256, 0, s>>>(p->stream_bhat, static_cast<float2*>(out), in.B, in.N, hop, c, out_len, c0, nb);
    FBST_CUDA_TRY(cudaGetLastError());
  }
  return FBST_OK;
}
