// C ABI of the FBST library (include/fbst.h): plan lifetime, memory, execution and status reporting.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <cmath>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "launch_util.cuh"

namespace fbst {

static thread_local char g_last_error[512] = "";

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s:%d)", cudaGetErrorName(e), what, file, line);
}

void set_last_error_message(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

struct mem_registry {
  std::unordered_map<void*, size_t> live;   // block -> bytes
};

int plan_alloc(fbst_plan_s* p, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) return FBST_OK;
  if (!p->mem) return FBST_ERR_INVALID;
  void* q = nullptr;
  if (p->alloc_fn) {
    q = p->alloc_fn(bytes, p->mem_stream, p->alloc_ctx);
    if (!q) {
      set_last_error_message("the plan's allocator returned NULL");
      return FBST_ERR_OOM;
    }
    if (reinterpret_cast<uintptr_t>(q) & 15u) {
      p->free_fn(q, bytes, p->mem_stream, p->alloc_ctx);
      set_last_error_message("the plan's allocator returned a block that is not 16-byte aligned");
      return FBST_ERR_INVALID;
    }
  } else {
    const cudaError_t e = cudaMallocAsync(&q, bytes, p->mem_stream);
    if (e != cudaSuccess) {
      set_last_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? FBST_ERR_OOM : FBST_ERR_CUDA;
    }
  }
  try {
    p->mem->live.emplace(q, bytes);
  } catch (...) {
    if (p->free_fn) p->free_fn(q, bytes, p->mem_stream, p->alloc_ctx);
    else cudaFreeAsync(q, p->mem_stream);
    return FBST_ERR_OOM;
  }
  *out = q;
  return FBST_OK;
}

void plan_free(fbst_plan_s* p, void* q) {
  if (!q || !p->mem) return;
  auto it = p->mem->live.find(q);
  if (it == p->mem->live.end()) return;
  const size_t bytes = it->second;
  p->mem->live.erase(it);
  if (p->free_fn) p->free_fn(q, bytes, p->mem_stream, p->alloc_ctx);
  else cudaFreeAsync(q, p->mem_stream);
}

// Every block still registered (the plan's own and those of nulling objects built on it).
static void free_plan_memory(fbst_plan_s* p) {
  if (!p->mem) return;
  while (!p->mem->live.empty()) plan_free(p, p->mem->live.begin()->first);
}

template <typename T>
static int dmalloc(fbst_plan_s* p, T** ptr, size_t count) {
  return plan_alloc_n(p, ptr, count);
}

static bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

int run_stage2(const fbst_plan_s* p, const float2* w, float2* bhat, int nb, cudaStream_t s, bool w_from_stage1) {
  switch (p->info.stage2) {
    case FBST_STAGE2_GS:
    case FBST_STAGE2_GS_IR1: return launch_stage2_gs(p, w, bhat, nb, s);
    case FBST_STAGE2_DENSE_FP32: return launch_stage2_dense_fp32(p, w, bhat, nb, s);
    case FBST_STAGE2_DENSE_BF16X3:
    case FBST_STAGE2_DENSE_TF32:
    case FBST_STAGE2_DENSE_TF32X3:
    case FBST_STAGE2_DENSE_F16X3: return launch_stage2_dense_tc(p, w, bhat, nb, s, w_from_stage1 && p->tc_wmax_stage1);
    default: return FBST_ERR_INVALID;
  }
}

static int check_exec_args(fbst_plan_s* p, const void* in, void* out, int nblk) {
  if (!p || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!in || !out || !aligned16(in) || !aligned16(out)) return FBST_ERR_INVALID;
  return FBST_OK;
}

#define FBST_TRY(expr)          \
  do {                          \
    const int fbst_r_ = (expr); \
    if (fbst_r_ != FBST_OK) return fbst_r_; \
  } while (0)

}  // namespace fbst

using namespace fbst;

extern "C" {

const char* fbst_status_string(int status) {
  switch (status) {
    case FBST_OK: return "FBST_OK";
    case FBST_ERR_INVALID: return "FBST_ERR_INVALID: a size, pointer or parameter is out of range";
    case FBST_ERR_OOM: return "FBST_ERR_OOM: allocation failed";
    case FBST_ERR_CUDA: return "FBST_ERR_CUDA: a CUDA call failed";
    case FBST_ERR_UNSUPPORTED: return "FBST_ERR_UNSUPPORTED: valid but not supported by this library";
    case FBST_ERR_TIMEOUT: return "FBST_ERR_TIMEOUT: a bounded device wait gave up";
    case FBST_ERR_NUMERIC: return "FBST_ERR_NUMERIC: a Toeplitz system is not numerically positive definite";
    default: return "unknown fbst status";
  }
}

const char* fbst_last_error(void) { return g_last_error; }

int fbst_plan_positions(fbst_plan_t* out, const fbst_geometry* g, const double* positions, int M, int N, int B,
                        const fbst_band* band, void* stream, fbst_alloc_fn alloc, fbst_free_fn free_fn, void* ctx) {
  if (!out) return FBST_ERR_INVALID;
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr)) return FBST_ERR_INVALID;
  fbst_info info;
  FBST_TRY(fbst_derive(g, M, N, B, band, &info));
  if (g->kind == FBST_URA && !positions && info.P_space_x != info.P_space_y) return FBST_ERR_UNSUPPORTED;
  // Elements off the grid: stage 1b becomes a type-1 NUFFT onto an oversampled grid of nf >= 2B
  // points (a linear array), or of nf_x x nf_y >= 2 bx x 2 by points (a rectangular array); the
  // grid sizes replace the chirp-z sizes in info.P_space_x / P_space_y.
  int nu_nf = 0, nu_nfy = 0;
  const int nu_w = 9;
  if (positions) {
    for (int m = 0; m < M; ++m)
      if (!std::isfinite(positions[2 * m]) || !std::isfinite(positions[2 * m + 1])) return FBST_ERR_INVALID;
    const size_t c64 = sizeof(float2), L = info.L;
    info.table_bytes -= c64 * L * ((size_t)g->mx + info.P_space_x + g->bx);
    if (g->kind == FBST_ULA) {
      for (int m = 0; m < M; ++m)
        if (positions[2 * m + 1] != 0.0) return FBST_ERR_INVALID;
      nu_nf = 16;
      while (nu_nf < 2 * B) nu_nf <<= 1;
      if (nu_nf > kMaxFFT) return FBST_ERR_UNSUPPORTED;
      info.table_bytes += sizeof(double) * M + (sizeof(int) + sizeof(float)) * L * M + sizeof(float) * B;
    } else {
      nu_nf = 16;
      while (nu_nf < 2 * g->bx) nu_nf <<= 1;
      nu_nfy = 16;
      while (nu_nfy < 2 * g->by) nu_nfy <<= 1;
      // The 2-D kernel's shared memory: the padded grid, the FFT exchange buffers, the [B][4 + 1]
      // output tile; grids up to 128 x 128.
      auto groups_x_nf = [](int nf) { return (size_t)256 / (nf / 2 < 32 ? nf / 2 : 32) * nf; };
      const size_t smem = sizeof(float) * 2 * nu_nf * ((size_t)nu_nfy + 1) +
                          c64 * (std::max(groups_x_nf(nu_nf), groups_x_nf(nu_nfy)) + (size_t)B * 5);
      if (nu_nf > 128 || nu_nfy > 128 || smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
      if (!(g->mx == g->my && g->bx == g->by))
        info.table_bytes -= c64 * L * ((size_t)g->my + info.P_space_y + g->by);
      info.table_bytes += 2 * (sizeof(double) * M + (sizeof(int) + sizeof(float)) * L * M) +
                          sizeof(float) * ((size_t)g->bx + g->by);
      info.P_space_y = nu_nfy;
    }
    info.P_space_x = nu_nf;
  }
  fbst_plan_s* p = new (std::nothrow) fbst_plan_s();
  if (!p) return FBST_ERR_OOM;
  std::memset(p, 0, sizeof(*p));
  p->mem = new (std::nothrow) mem_registry();
  if (!p->mem) {
    delete p;
    return FBST_ERR_OOM;
  }
  p->info = info;
  p->geom = *g;
  p->band = *band;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  p->alloc_fn = alloc;
  p->free_fn = free_fn;
  p->alloc_ctx = ctx;
  p->mem_stream = s;
  p->nu_nf = nu_nf;
  p->nu_nfy = nu_nfy;
  p->nu_w = nu_nf ? nu_w : 0;
  int r = FBST_OK;
  do {
    if (cudaGetDevice(&p->device) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    const int L = info.L;
    if ((r = dmalloc(p, &p->tw32, kTwiddleSize)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->tw64, kTwiddleSize)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->pre_t, info.N)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->gspec_t, (size_t)info.S_time * info.P_time)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->post_t, L)) != FBST_OK) break;
    p->ax[0] = fbst_axis_tables{g->mx, g->bx, info.P_space_x, nullptr, nullptr, nullptr};
    p->n_axes = 1;
    p->same_axes = 1;
    if (g->kind == FBST_URA) {
      p->ax[1] = fbst_axis_tables{g->my, g->by, info.P_space_y, nullptr, nullptr, nullptr};
      if (!(g->mx == g->my && g->bx == g->by)) {
        p->n_axes = 2;
        p->same_axes = 0;
      }
    }
    if (nu_nf) {
      if ((r = dmalloc(p, &p->pos, (size_t)M)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->nu_j0, (size_t)L * M)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->nu_dg, (size_t)L * M)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->nu_deconv, (size_t)(nu_nfy ? g->bx : B))) != FBST_OK) break;
      if (nu_nfy) {
        if ((r = dmalloc(p, &p->pos_y, (size_t)M)) != FBST_OK) break;
        if ((r = dmalloc(p, &p->nu_j0y, (size_t)L * M)) != FBST_OK) break;
        if ((r = dmalloc(p, &p->nu_dgy, (size_t)L * M)) != FBST_OK) break;
        if ((r = dmalloc(p, &p->nu_deconv_y, (size_t)g->by)) != FBST_OK) break;
      }
      std::vector<double> px(M), py(M);
      for (int m = 0; m < M; ++m) {
        px[m] = positions[2 * m];
        py[m] = positions[2 * m + 1];
      }
      if (cudaStreamSynchronize(s) != cudaSuccess ||
          cudaMemcpy(p->pos, px.data(), sizeof(double) * M, cudaMemcpyHostToDevice) != cudaSuccess ||
          (nu_nfy && cudaMemcpy(p->pos_y, py.data(), sizeof(double) * M, cudaMemcpyHostToDevice) != cudaSuccess)) {
        r = FBST_ERR_CUDA;
        break;
      }
    }
    for (int a = 0; a < (nu_nf ? 0 : p->n_axes) && r == FBST_OK; ++a) {
      fbst_axis_tables& ax = p->ax[a];
      if ((r = dmalloc(p, &ax.pre, (size_t)L * ax.Ma)) != FBST_OK) break;
      if ((r = dmalloc(p, &ax.kspec, (size_t)L * ax.P)) != FBST_OK) break;
      if ((r = dmalloc(p, &ax.post, (size_t)L * ax.Ba)) != FBST_OK) break;
    }
    if (r != FBST_OK) break;
    if (p->same_axes && g->kind == FBST_URA) {
      p->ax[1].pre = p->ax[0].pre;
      p->ax[1].kspec = p->ax[0].kspec;
      p->ax[1].post = p->ax[0].post;
    }
    if ((r = dmalloc(p, &p->x64, (size_t)B * L)) != FBST_OK) break;
    if (info.stage2 == FBST_STAGE2_GS || info.stage2 == FBST_STAGE2_GS_IR1) {
      if ((r = dmalloc(p, &p->XV, (size_t)B * 2 * info.P_gs)) != FBST_OK) break;
      if (info.stage2 == FBST_STAGE2_GS_IR1 && (r = dmalloc(p, &p->Aspec, (size_t)B * info.P_gs)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->pre_r, (size_t)L)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->qspec_r, (size_t)info.S_rec * info.P_rec)) != FBST_OK) break;
      if ((r = dmalloc(p, &p->post_r, (size_t)info.N)) != FBST_OK) break;
    } else {
      if ((r = dmalloc(p, &p->G, (size_t)B * info.N * L)) != FBST_OK) break;
    }
    if ((r = dmalloc(p, &p->ws_yhat, (size_t)band->max_blocks * L * M)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->ws_w, (size_t)band->max_blocks * B * L)) != FBST_OK) break;
    if ((r = dmalloc(p, &p->d_status, 1)) != FBST_OK) break;
    if (cudaMemsetAsync(p->d_status, 0, sizeof(int), s) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    r = build_plan_tables(p, s);
  } while (0);
  if (r != FBST_OK) {
    cudaStreamSynchronize(s);
    free_plan_memory(p);
    cudaStreamSynchronize(s);
    delete p->mem;
    delete p;
    return r;
  }
  *out = p;
  return FBST_OK;
}

int fbst_plan(fbst_plan_t* out, const fbst_geometry* g, int M, int N, int B, const fbst_band* band, void* stream,
              fbst_alloc_fn alloc, fbst_free_fn free_fn, void* ctx) {
  return fbst_plan_positions(out, g, nullptr, M, N, B, band, stream, alloc, free_fn, ctx);
}

static void free_trace(fbst_plan_s* p);

int fbst_destroy(fbst_plan_t p) {
  if (!p) return FBST_OK;
  // The host path's copy streams hold no pending work: fbst_execute_host synchronises before it
  // returns. The frees are ordered on the plan's stream.
  for (cudaStream_t c : {p->copy_in, p->copy_out})
    if (c) cudaStreamDestroy(c);
  for (cudaEvent_t e : p->pipe_ev)
    if (e) cudaEventDestroy(e);
  free_trace(p);
  free_plan_memory(p);
  delete p->mem;
  delete p;
  return FBST_OK;
}

int fbst_sync_status(fbst_plan_t p, void* stream) {
  if (!p) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  FBST_CUDA_TRY(cudaStreamSynchronize(s));
  int st = 0;
  FBST_CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) FBST_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)));
  return st;
}

int fbst_set_wait_limit(fbst_plan_t p, uint64_t ns) {
  if (!p) return FBST_ERR_INVALID;
  p->wait_ns = ns;
  return FBST_OK;
}

int fbst_plan_info(fbst_plan_t p, fbst_info* out) {
  if (!p || !out) return FBST_ERR_INVALID;
  *out = p->info;
  return FBST_OK;
}

int fbst_plan_generators(fbst_plan_t p, void* x_host) {
  if (!p || !x_host) return FBST_ERR_INVALID;
  FBST_CUDA_TRY(cudaMemcpy(x_host, p->x64, sizeof(double2) * (size_t)p->info.B * p->info.L, cudaMemcpyDeviceToHost));
  return FBST_OK;
}

int fbst_solve_generators(fbst_plan_t p, int method, void* x, void* stream) {
  if (!p || !x) return FBST_ERR_INVALID;
  if (method != FBST_GEN_LEVINSON && method != FBST_GEN_SUPERFAST) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double2* gen = nullptr;
  FBST_TRY(plan_alloc_n(p, &gen, (size_t)p->info.B * p->info.L));
  const bool other = s != p->mem_stream;  // allocated in stream order on the plan's stream
  int r = (other && cudaStreamSynchronize(p->mem_stream) != cudaSuccess) ? FBST_ERR_CUDA : FBST_OK;
  if (r == FBST_OK) r = plan_toeplitz_generators(p, gen, s);
  if (r == FBST_OK) r = solve_generators(p, gen, static_cast<double2*>(x), p->info.B, method, s);
  if (other) cudaStreamSynchronize(s);
  plan_free(p, gen);
  return r;
}

int fbst_czt_time(fbst_plan_t p, const void* y, void* yhat, int nblk, void* stream) {
  FBST_TRY(check_exec_args(p, y, yhat, nblk));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  for (int c0 = 0; c0 < nblk; c0 += 65535) {
    const int nb = std::min(65535, nblk - c0);
    FBST_TRY(launch_czt_time(p, static_cast<const float2*>(y) + (size_t)c0 * in.M * in.N,
                             static_cast<float2*>(yhat) + (size_t)c0 * in.L * in.M, nb, s));
  }
  return FBST_OK;
}

int fbst_czt_space(fbst_plan_t p, const void* yhat, void* w, int nblk, void* stream) {
  FBST_TRY(check_exec_args(p, yhat, w, nblk));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  for (int c0 = 0; c0 < nblk; c0 += 65535) {
    const int nb = std::min(65535, nblk - c0);
    FBST_TRY(launch_czt_space(p, static_cast<const float2*>(yhat) + (size_t)c0 * in.L * in.M,
                              static_cast<float2*>(w) + (size_t)c0 * in.B * in.L, nb, s));
  }
  return FBST_OK;
}

int fbst_czt(fbst_plan_t p, const void* y, void* w, int nblk, void* stream) {
  FBST_TRY(check_exec_args(p, y, w, nblk));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  const int maxb = p->band.max_blocks;
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(launch_czt_time(p, static_cast<const float2*>(y) + (size_t)c0 * in.M * in.N, p->ws_yhat, nb, s));
    FBST_TRY(launch_czt_space(p, p->ws_yhat, static_cast<float2*>(w) + (size_t)c0 * in.B * in.L, nb, s));
  }
  return FBST_OK;
}

int fbst_toeplitz_apply(fbst_plan_t p, const void* w, void* bhat, int nblk, void* stream) {
  FBST_TRY(check_exec_args(p, w, bhat, nblk));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  const int maxb = p->band.max_blocks;
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(run_stage2(p, static_cast<const float2*>(w) + (size_t)c0 * in.B * in.L,
                        static_cast<float2*>(bhat) + (size_t)c0 * in.B * in.N, nb, s));
  }
  return FBST_OK;
}

int fbst_execute(fbst_plan_t p, const void* y, void* bhat, int nblk, void* stream) {
  FBST_TRY(check_exec_args(p, y, bhat, nblk));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  const int maxb = p->band.max_blocks;
  // Traced call: events around the three stages of its first chunk.
  cudaEvent_t* tev = nullptr;
  if (p->trace_cap > 0 && nblk > 0) {
    tev = p->trace_ev + 4 * (size_t)(p->trace_next % p->trace_cap);
    ++p->trace_next;
    p->trace_count = std::min(p->trace_count + 1, p->trace_cap);
  }
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    cudaEvent_t* ev = c0 == 0 ? tev : nullptr;
    if (ev) FBST_CUDA_TRY(cudaEventRecord(ev[0], s));
    FBST_TRY(launch_czt_time(p, static_cast<const float2*>(y) + (size_t)c0 * in.M * in.N, p->ws_yhat, nb, s));
    if (ev) FBST_CUDA_TRY(cudaEventRecord(ev[1], s));
    FBST_TRY(launch_czt_space_scaled(p, p->ws_yhat, p->ws_w, nb, 0, s));
    if (ev) FBST_CUDA_TRY(cudaEventRecord(ev[2], s));
    FBST_TRY(run_stage2(p, p->ws_w, static_cast<float2*>(bhat) + (size_t)c0 * in.B * in.N, nb, s, true));
    if (ev) FBST_CUDA_TRY(cudaEventRecord(ev[3], s));
  }
  return FBST_OK;
}

static void free_trace(fbst_plan_s* p) {
  for (int i = 0; i < 4 * p->trace_cap; ++i)
    if (p->trace_ev[i]) cudaEventDestroy(p->trace_ev[i]);
  delete[] p->trace_ev;
  p->trace_ev = nullptr;
  p->trace_cap = p->trace_next = p->trace_count = 0;
}

int fbst_trace_stages(fbst_plan_t p, int capacity) {
  if (!p || capacity < 0 || capacity > (1 << 20)) return FBST_ERR_INVALID;
  free_trace(p);
  if (capacity == 0) return FBST_OK;
  p->trace_ev = new (std::nothrow) cudaEvent_t[4 * (size_t)capacity]();
  if (!p->trace_ev) return FBST_ERR_OOM;
  p->trace_cap = capacity;
  for (int i = 0; i < 4 * capacity; ++i) {
    const cudaError_t e = cudaEventCreate(&p->trace_ev[i]);
    if (e != cudaSuccess) {
      p->trace_ev[i] = nullptr;
      free_trace(p);
      set_last_cuda_error(e, "cudaEventCreate", __FILE__, __LINE__);
      return FBST_ERR_CUDA;
    }
  }
  return FBST_OK;
}

int fbst_trace_read(fbst_plan_t p, float* ms, int max_calls) {
  if (!p || (!ms && max_calls > 0) || max_calls < 0) return FBST_ERR_INVALID;
  const int n = std::min(p->trace_count, max_calls);
  const int first = p->trace_next - p->trace_count;  // the oldest call not yet read
  for (int i = 0; i < n; ++i) {
    cudaEvent_t* ev = p->trace_ev + 4 * (size_t)((first + i) % p->trace_cap);
    FBST_CUDA_TRY(cudaEventSynchronize(ev[3]));
    for (int j = 0; j < 3; ++j) FBST_CUDA_TRY(cudaEventElapsedTime(&ms[3 * i + j], ev[j], ev[j + 1]));
  }
  p->trace_count = 0;
  return n;
}

}  // extern "C"

namespace fbst {

// One chunk (at most max_blocks blocks) of fbst_execute_host with the copies overlapped with the
// kernels: the input moves in up to 4 block parts on the copy_in stream while stage 1 of the
// previous part runs on s; stage 2 then runs in up to 4 parts, each part's output moving out on
// the copy_out stream while the next part computes. (Alternating the parts over two streams per
// direction was measured slower: concurrent copies in one direction contend.) The stage-2 parts are beam ranges for the
// TF32x3 tensor-core operator (each part of G is read once) and block parts for the
// Gohberg-Semencul variants; the other dense variants run stage 2 once (a block split would read G
// once per part). With a pinned output, stage 2 runs once and stores into it directly. s is left
// ordered after the outgoing copies.
// bh_dev: the device address of bh when the caller's output is pinned (mapped) host memory, else
// null. Stage 2 then stores straight into it and no output copy is needed.
static int execute_host_chunk(fbst_plan_s* p, const char* yh, char* bh, float2* bh_dev, int nb, cudaStream_t s) {
  const fbst_info& in = p->info;
  cudaEvent_t* ev = p->pipe_ev;
  const size_t yblk = (size_t)in.M * in.N, hblk = (size_t)in.L * in.M, wblk = (size_t)in.B * in.L,
               bblk = (size_t)in.B * in.N;
  const bool direct = bh_dev != nullptr;
  const bool gs = !direct && (in.stage2 == FBST_STAGE2_GS || in.stage2 == FBST_STAGE2_GS_IR1);
  const bool beam_parts =
      !direct && (in.stage2 == FBST_STAGE2_DENSE_TF32X3 || in.stage2 == FBST_STAGE2_DENSE_F16X3);
  // Everything earlier on s (including the previous chunk's reads of stage_y) precedes the copies in.
  FBST_CUDA_TRY(cudaEventRecord(ev[0], s));
  FBST_CUDA_TRY(cudaStreamWaitEvent(p->copy_in, ev[0], 0));
  const int q1 = std::min(4, nb);
  for (int i = 0; i < q1; ++i) {
    const size_t a = (size_t)nb * i / q1, e = (size_t)nb * (i + 1) / q1;
    cudaStream_t ci = p->copy_in;
    FBST_CUDA_TRY(cudaMemcpyAsync(p->stage_y + a * yblk, yh + sizeof(float2) * a * yblk, sizeof(float2) * (e - a) * yblk,
                                  cudaMemcpyHostToDevice, ci));
    FBST_CUDA_TRY(cudaEventRecord(ev[1 + i], ci));
    FBST_CUDA_TRY(cudaStreamWaitEvent(s, ev[1 + i], 0));
    FBST_TRY(launch_czt_time(p, p->stage_y + a * yblk, p->ws_yhat + a * hblk, (int)(e - a), s));
    FBST_TRY(launch_czt_space_scaled(p, p->ws_yhat + a * hblk, p->ws_w + a * wblk, (int)(e - a), (int)a, s));
    if (gs) {
      FBST_TRY(run_stage2(p, p->ws_w + a * wblk, p->stage_bhat + a * bblk, (int)(e - a), s));
      FBST_CUDA_TRY(cudaEventRecord(ev[5 + i], s));
      FBST_CUDA_TRY(cudaStreamWaitEvent(p->copy_out, ev[5 + i], 0));
      FBST_CUDA_TRY(cudaMemcpyAsync(bh + sizeof(float2) * a * bblk, p->stage_bhat + a * bblk,
                                    sizeof(float2) * (e - a) * bblk, cudaMemcpyDeviceToHost, p->copy_out));
    }
  }
  if (beam_parts) {
    // One set of block scales for every beam range (already written by stage 1b on a grid array).
    if (!p->tc_wmax_stage1) FBST_TRY(prepare_dense_tc_scales(p, p->ws_w, nb, s));
    const int q2 = std::min(4, in.B);
    for (int r = 0; r < q2; ++r) {
      const int b0 = in.B * r / q2, b1 = in.B * (r + 1) / q2;
      FBST_TRY(launch_stage2_dense_tc_beams(p, p->ws_w, p->stage_bhat, nb, b0, b1 - b0, s));
      FBST_CUDA_TRY(cudaEventRecord(ev[5 + r], s));
      FBST_CUDA_TRY(cudaStreamWaitEvent(p->copy_out, ev[5 + r], 0));
      // bhat [nb][B][N]: beams [b0, b1) of every block, a strided 2-D copy.
      const size_t pitch = sizeof(float2) * bblk;
      FBST_CUDA_TRY(cudaMemcpy2DAsync(bh + sizeof(float2) * (size_t)b0 * in.N, pitch, p->stage_bhat + (size_t)b0 * in.N,
                                      pitch, sizeof(float2) * (size_t)(b1 - b0) * in.N, nb, cudaMemcpyDeviceToHost,
                                      p->copy_out));
    }
  } else if (direct) {
    FBST_TRY(run_stage2(p, p->ws_w, bh_dev, nb, s, true));
    return FBST_OK;
  } else if (!gs) {
    FBST_TRY(run_stage2(p, p->ws_w, p->stage_bhat, nb, s, true));
    FBST_CUDA_TRY(cudaEventRecord(ev[5], s));
    FBST_CUDA_TRY(cudaStreamWaitEvent(p->copy_out, ev[5], 0));
    FBST_CUDA_TRY(cudaMemcpyAsync(bh, p->stage_bhat, sizeof(float2) * (size_t)nb * bblk, cudaMemcpyDeviceToHost,
                                  p->copy_out));
  }
  FBST_CUDA_TRY(cudaEventRecord(ev[9], p->copy_out));
  FBST_CUDA_TRY(cudaStreamWaitEvent(s, ev[9], 0));
  return FBST_OK;
}

}  // namespace fbst

extern "C" {

int fbst_execute_host(fbst_plan_t p, const void* y_host, void* bhat_host, int nblk, void* stream) {
  if (!p || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!y_host || !bhat_host) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = p->info;
  const int maxb = p->band.max_blocks;
  if (!p->stage_y || !p->stage_bhat) {
    if (!p->stage_y) FBST_TRY(dmalloc(p, &p->stage_y, (size_t)maxb * in.M * in.N));
    if (!p->stage_bhat) FBST_TRY(dmalloc(p, &p->stage_bhat, (size_t)maxb * in.B * in.N));
    // The staging blocks were allocated in stream order on the plan's stream; make them usable
    // on the copy streams and `stream` (once).
    FBST_CUDA_TRY(cudaStreamSynchronize(p->mem_stream));
  }
  for (cudaStream_t* c : {&p->copy_in, &p->copy_out})
    if (!*c) FBST_CUDA_TRY(cudaStreamCreateWithFlags(c, cudaStreamNonBlocking));
  for (cudaEvent_t& e : p->pipe_ev)
    if (!e) FBST_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // Pinned output: stage 2 writes it in place through its device address (unified addressing).
  float2* bh_dev = nullptr;
  {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, bhat_host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer)
      bh_dev = static_cast<float2*>(at.devicePointer);
    cudaGetLastError();
  }
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(execute_host_chunk(p, static_cast<const char*>(y_host) + sizeof(float2) * (size_t)c0 * in.M * in.N,
                                static_cast<char*>(bhat_host) + sizeof(float2) * (size_t)c0 * in.B * in.N,
                                bh_dev ? bh_dev + (size_t)c0 * in.B * in.N : nullptr, nb, s));
  }
  FBST_CUDA_TRY(cudaStreamSynchronize(s));
  return FBST_OK;
}

int fbst_launch_count(fbst_plan_t p, int nblk) {
  if (!p || nblk <= 0) return 0;
  const int chunks = (nblk + p->band.max_blocks - 1) / p->band.max_blocks;
  return chunks * (2 + stage2_launches(p, true));
}

}  // extern "C"
