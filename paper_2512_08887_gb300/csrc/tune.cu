// Autotuner of the Stockham launch shapes (elements per thread = radix, transforms per CTA) of
// the two stage-1 kernels. For a plan and a block count it times every compiled shape of the
// temporal and the spatial chirp-z with CUDA events on the plan's own workspace and keeps the
// fastest in the plan. The Python layer (autotune.py) caches the choice per problem size in JSON.
#include <cfloat>
#include <cstring>

#include "common.cuh"
#include "launch_util.cuh"

namespace fbst {

template <typename F>
static int time_variant(F&& launch, cudaStream_t s, float* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  FBST_CUDA_TRY(cudaEventCreate(&a));
  FBST_CUDA_TRY(cudaEventCreate(&b));
  int r = launch();  // warm-up (and one-time set-up)
  if (r == FBST_OK) {
    cudaEventRecord(a, s);
    for (int k = 0; k < 5 && r == FBST_OK; ++k) r = launch();
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *ms_out = ms / 5.f;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return r;
}

}  // namespace fbst

using namespace fbst;

extern "C" {

int fbst_set_shapes(fbst_plan_t p, int time_E, int time_G, int space_E, int space_G) {
  if (!p) return FBST_ERR_INVALID;
  auto valid = [](int (*list)(int, fft_shape*, int), int P, int E, int G) {
    if (E == 0 && G == 0) return true;
    fft_shape all[16];
    const int n = list(P, all, 16);
    for (int i = 0; i < n; ++i)
      if (all[i].E == E && all[i].G == G) return true;
    return false;
  };
  if (!valid(time_shapes, p->info.P_time, time_E, time_G)) return FBST_ERR_UNSUPPORTED;
  if (!valid(space_shapes, p->info.P_space_x, space_E, space_G)) return FBST_ERR_UNSUPPORTED;
  p->shape_time = fft_shape{time_E, time_G};
  p->shape_space = fft_shape{space_E, space_G};
  return FBST_OK;
}

int fbst_get_shapes(fbst_plan_t p, int* shapes4) {
  if (!p || !shapes4) return FBST_ERR_INVALID;
  const fft_shape t = time_shape(p), sp = space_shape(p);
  shapes4[0] = t.E;
  shapes4[1] = t.G;
  shapes4[2] = sp.E;
  shapes4[3] = sp.G;
  return FBST_OK;
}

int fbst_autotune(fbst_plan_t p, int nblk, void* stream, int* shapes4) {
  if (!p || nblk < 1 || nblk > p->band.max_blocks) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  float2* y = nullptr;
  {
    const int ra = plan_alloc_n(p, &y, (size_t)nblk * in.M * in.N);
    if (ra != FBST_OK) return ra;
  }
  FBST_CUDA_TRY(cudaStreamSynchronize(p->mem_stream));   // allocated in order on the plan's stream
  FBST_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(float2) * (size_t)nblk * in.M * in.N, s));
  int r = FBST_OK;
  // Temporal chirp-z.
  {
    fft_shape all[16];
    const int n = time_shapes(in.P_time, all, 16);
    float best = FLT_MAX;
    fft_shape pick = time_shape(p);
    for (int i = 0; i < n && r == FBST_OK; ++i) {
      p->shape_time = all[i];
      float ms = FLT_MAX;
      const int ri = time_variant([&] { return launch_czt_time(p, y, p->ws_yhat, nblk, s); }, s, &ms);
      if (ri == FBST_OK && ms < best) {
        best = ms;
        pick = all[i];
      } else if (ri != FBST_OK && ri != FBST_ERR_UNSUPPORTED) {
        r = ri;
      }
    }
    p->shape_time = pick;
  }
  // Spatial chirp-z (linear arrays).
  if (r == FBST_OK && p->geom.kind == FBST_ULA && !p->nu_nf) {
    fft_shape all[16];
    const int n = space_shapes(in.P_space_x, all, 16);
    float best = FLT_MAX;
    fft_shape pick = space_shape(p);
    for (int i = 0; i < n && r == FBST_OK; ++i) {
      p->shape_space = all[i];
      float ms = FLT_MAX;
      const int ri = time_variant([&] { return launch_czt_space(p, p->ws_yhat, p->ws_w, nblk, s); }, s, &ms);
      if (ri == FBST_OK && ms < best) {
        best = ms;
        pick = all[i];
      } else if (ri != FBST_OK && ri != FBST_ERR_UNSUPPORTED) {
        r = ri;
      }
    }
    p->shape_space = pick;
  }
  cudaStreamSynchronize(s);
  plan_free(p, y);
  if (r == FBST_OK && shapes4) r = fbst_get_shapes(p, shapes4);
  return r;
}

}  // extern "C"
