// Batches of independent plans (uneven arrays: different M, N, B, fb) executed as a few fused
// launches and replayed as a CUDA graph.
//
// A batch run groups its plans' work by kernel and transform size: every temporal chirp-z job with
// the same (P_time, launch shape) goes into one launch, likewise the spatial chirp-z jobs and the
// stage-2 jobs with the same (P_gs, P_rec, S_rec, refinement). Each launch spreads the flattened
// work items of all its jobs evenly over the resident CTAs, so small arrays fill the GPU together
// instead of one at a time. The launch sequence of a given set of pointers and block counts is
// captured once into a CUDA graph (on an internal stream) and replayed on the caller's stream.
#include <algorithm>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "launch_util.cuh"

struct fbst_batch_s {
  std::vector<fbst_plan_s*> plans;
  // Graph of the last configuration.
  std::vector<const void*> key_y;
  std::vector<void*> key_bhat;
  std::vector<int> key_nblk;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  int launches = 0;
};

namespace fbst {

// Enqueue every launch of one batch run on stream s; returns the number of kernels launched.
static int enqueue_batch(fbst_batch_s* bt, const void* const* y, void* const* bhat, const int* nblk, cudaStream_t s,
                         int* launches) {
  *launches = 0;
  const int n = (int)bt->plans.size();
  // ---- temporal chirp-z, grouped by (P, E, G)
  {
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
      if (nblk[i] <= 0) continue;
      const fft_shape sh = time_shape(bt->plans[i]);
      groups[{bt->plans[i]->info.P_time, sh.E, sh.G}].push_back(i);
    }
    for (auto& kv : groups) {
      const int P = std::get<0>(kv.first);
      const fft_shape sh{std::get<1>(kv.first), std::get<2>(kv.first)};
      const std::vector<int>& ids = kv.second;
      for (size_t c0 = 0; c0 < ids.size(); c0 += kMaxJobs) {
        job_list<time_job> jl;
        jl.n = 0;
        jl.total = 0;
        int max_Lh = 0;
        for (size_t k = c0; k < std::min(ids.size(), c0 + kMaxJobs); ++k) {
          fbst_plan_s* p = bt->plans[ids[k]];
          time_job j = make_time_job(p, static_cast<const float2*>(y[ids[k]]), p->ws_yhat, nblk[ids[k]]);
          j.first = jl.total;
          jl.total += time_items(j, sh, P);
          jl.job[jl.n++] = j;
          max_Lh = std::max(max_Lh, p->info.L / p->info.S_time);
        }
        FBST_TRY(launch_time_jobs(jl, P, sh, max_Lh, bt->plans[ids[c0]]->tw32, s));
        ++*launches;
      }
    }
  }
  // ---- spatial chirp-z: linear arrays grouped by (P, E, G); rectangular and non-uniform arrays one by one
  {
    std::map<std::tuple<int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
      if (nblk[i] <= 0) continue;
      fbst_plan_s* p = bt->plans[i];
      if (p->geom.kind != FBST_ULA || p->nu_nf) {
        FBST_TRY(launch_czt_space(p, p->ws_yhat, p->ws_w, nblk[i], s));
        ++*launches;
        continue;
      }
      const fft_shape sh = space_shape(p);
      groups[{p->info.P_space_x, sh.E, sh.G}].push_back(i);
    }
    for (auto& kv : groups) {
      const int P = std::get<0>(kv.first);
      const fft_shape sh{std::get<1>(kv.first), std::get<2>(kv.first)};
      const std::vector<int>& ids = kv.second;
      for (size_t c0 = 0; c0 < ids.size(); c0 += kMaxJobs) {
        job_list<space_job> jl;
        jl.n = 0;
        jl.total = 0;
        int max_B = 0;
        for (size_t k = c0; k < std::min(ids.size(), c0 + kMaxJobs); ++k) {
          fbst_plan_s* p = bt->plans[ids[k]];
          space_job j = make_space_job(p, p->ws_yhat, p->ws_w, nblk[ids[k]]);
          j.first = jl.total;
          jl.total += space_items(j, sh, P);
          jl.job[jl.n++] = j;
          max_B = std::max(max_B, p->ax[0].Ba);
        }
        FBST_TRY(launch_space_jobs(jl, P, sh, max_B, bt->plans[ids[c0]]->tw32, s));
        ++*launches;
      }
    }
  }
  // ---- stage 2: GS variants grouped by (P_gs, P_rec, S_rec, refinement); dense plans one by one
  {
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    for (int i = 0; i < n; ++i) {
      if (nblk[i] <= 0) continue;
      fbst_plan_s* p = bt->plans[i];
      const int k = p->info.stage2;
      if (k == FBST_STAGE2_GS || k == FBST_STAGE2_GS_IR1) {
        groups[{p->info.P_gs, p->info.P_rec, p->info.S_rec, k == FBST_STAGE2_GS_IR1}].push_back(i);
      } else if (k == FBST_STAGE2_DENSE_FP32) {
        FBST_TRY(launch_stage2_dense_fp32(p, p->ws_w, static_cast<float2*>(bhat[i]), nblk[i], s));
        ++*launches;
      } else {
        FBST_TRY(launch_stage2_dense_tc(p, p->ws_w, static_cast<float2*>(bhat[i]), nblk[i], s));
        *launches += 2;
      }
    }
    for (auto& kv : groups) {
      const int PG = std::get<0>(kv.first), PR = std::get<1>(kv.first), SR = std::get<2>(kv.first);
      const bool IR = std::get<3>(kv.first) != 0;
      const std::vector<int>& ids = kv.second;
      for (size_t c0 = 0; c0 < ids.size(); c0 += kMaxJobs) {
        job_list<gs_job> jl;
        jl.n = 0;
        jl.total = 0;
        int max_L = 0;
        for (size_t k = c0; k < std::min(ids.size(), c0 + kMaxJobs); ++k) {
          fbst_plan_s* p = bt->plans[ids[k]];
          gs_job j = make_gs_job(p, p->ws_w, static_cast<float2*>(bhat[ids[k]]), nblk[ids[k]]);
          j.first = jl.total;
          jl.total += (long long)p->info.B * nblk[ids[k]];
          jl.job[jl.n++] = j;
          max_L = std::max(max_L, p->info.L);
        }
        FBST_TRY(launch_gs_jobs(jl, PG, PR, SR, IR, max_L, bt->plans[ids[c0]]->tw32, s));
        ++*launches;
      }
    }
  }
  return FBST_OK;
}

static void drop_graph(fbst_batch_s* bt) {
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  bt->exec = nullptr;
  bt->graph = nullptr;
  bt->key_y.clear();
  bt->key_bhat.clear();
  bt->key_nblk.clear();
}

}  // namespace fbst

using namespace fbst;

extern "C" {

int fbst_batch_create(fbst_batch_t* out, const fbst_plan_t* plans, int count) {
  if (!out || !plans || count < 1) return FBST_ERR_INVALID;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!plans[i]) return FBST_ERR_INVALID;
    for (int k = 0; k < i; ++k)
      if (plans[k] == plans[i]) return FBST_ERR_INVALID;  // each plan's workspace serves one job
  }
  fbst_batch_s* bt = new (std::nothrow) fbst_batch_s();
  if (!bt) return FBST_ERR_OOM;
  bt->plans.assign(plans, plans + count);
  if (cudaStreamCreateWithFlags(&bt->capture, cudaStreamNonBlocking) != cudaSuccess) {
    delete bt;
    return FBST_ERR_CUDA;
  }
  *out = bt;
  return FBST_OK;
}

int fbst_batch_execute(fbst_batch_t bt, const void* const* y, void* const* bhat, const int* nblk, void* stream) {
  if (!bt || !y || !bhat || !nblk) return FBST_ERR_INVALID;
  const int n = (int)bt->plans.size();
  for (int i = 0; i < n; ++i) {
    if (nblk[i] < 0 || nblk[i] > bt->plans[i]->band.max_blocks) return FBST_ERR_INVALID;
    if (nblk[i] > 0 && (!y[i] || !bhat[i] || (reinterpret_cast<uintptr_t>(y[i]) & 15u) ||
                        (reinterpret_cast<uintptr_t>(bhat[i]) & 15u)))
      return FBST_ERR_INVALID;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool same = bt->exec && std::equal(bt->key_y.begin(), bt->key_y.end(), y) &&
                    std::equal(bt->key_bhat.begin(), bt->key_bhat.end(), bhat) &&
                    std::equal(bt->key_nblk.begin(), bt->key_nblk.end(), nblk);
  if (same) {
    FBST_CUDA_TRY(cudaGraphLaunch(bt->exec, s));
    return FBST_OK;
  }
  // New configuration: run it eagerly (this also performs every one-time kernel set-up), then
  // capture the same launch sequence into a graph for the following calls.
  drop_graph(bt);
  int launches = 0;
  FBST_TRY(enqueue_batch(bt, y, bhat, nblk, s, &launches));
  FBST_CUDA_TRY(cudaStreamBeginCapture(bt->capture, cudaStreamCaptureModeThreadLocal));
  int captured = 0;
  const int r = enqueue_batch(bt, y, bhat, nblk, bt->capture, &captured);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(bt->capture, &g);
  if (r != FBST_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return r != FBST_OK ? r : FBST_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return FBST_ERR_CUDA;
  }
  bt->graph = g;
  bt->exec = ex;
  bt->key_y.assign(y, y + n);
  bt->key_bhat.assign(bhat, bhat + n);
  bt->key_nblk.assign(nblk, nblk + n);
  bt->launches = captured;
  return FBST_OK;
}

int fbst_batch_enqueue(fbst_batch_t bt, const void* const* y, void* const* bhat, const int* nblk, void* stream) {
  if (!bt || !y || !bhat || !nblk) return FBST_ERR_INVALID;
  const int n = (int)bt->plans.size();
  for (int i = 0; i < n; ++i) {
    if (nblk[i] < 0 || nblk[i] > bt->plans[i]->band.max_blocks) return FBST_ERR_INVALID;
    if (nblk[i] > 0 && (!y[i] || !bhat[i] || (reinterpret_cast<uintptr_t>(y[i]) & 15u) ||
                        (reinterpret_cast<uintptr_t>(bhat[i]) & 15u)))
      return FBST_ERR_INVALID;
  }
  int launches = 0;
  return enqueue_batch(bt, y, bhat, nblk, reinterpret_cast<cudaStream_t>(stream), &launches);
}

int fbst_batch_launch_count(fbst_batch_t bt) { return bt ? bt->launches : 0; }

int fbst_batch_destroy(fbst_batch_t bt) {
  if (!bt) return FBST_OK;
  drop_graph(bt);
  if (bt->capture) {
    cudaStreamSynchronize(bt->capture);
    cudaStreamDestroy(bt->capture);
  }
  delete bt;
  return FBST_OK;
}

}  // extern "C"
