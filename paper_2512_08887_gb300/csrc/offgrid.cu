// Off-grid beams by interpolation of beam vectors (Sec. VIII-A), on top of an FBST plan.
//
// A direction (u, v) between the grid beams gets its beam vector w* from the stage-1 vectors w_b of
// the K grid beams around it along each axis (the paper uses 8): a natural cubic spline in the
// direction cosine (the grid is uniform in u, u_a = -1 + 2a/bx), evaluated at u, and for a
// rectangular array the tensor product of the splines along u and v. The spline is linear in the
// data, so w* = sum_i c_i w_{b_i} with weights fixed per direction; they are computed once on the
// host in FP64. The off-grid beam is then the regularised least-squares beam of that direction
// (Eq. (5)-(7)): bhat* = F_u A*^{-1} w*, with A* = F*^H F* + delta I of the off-grid direction itself,
// applied by Gohberg-Semencul with one refinement step (Sec. V) from FP64 plan-time spectra.
//
// Plan time: weights and windows (host, FP64); generators of every A* from their closed form, FP64
// Levinson, Gohberg-Semencul and circulant spectra, reconstruction tables (plan.cu, FP64, rounded
// once). Run time, per chunk of at most max_blocks blocks: k_offgrid_interp (w -> w*, FP32), then the
// stage-2 Gohberg-Semencul kernel of the plan through a descriptor whose beams are the directions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "launch_util.cuh"
#include "spline.cuh"

namespace fbst {
namespace {

// wstar[blk][k][ell] = sum_{i<Kx, j<Ky} cx[k][i] cy[k][j] w[blk][(ax_k + i)*by + ay_k + j][ell], two
// complex values (one float4) per thread; grid (ell pairs, direction, block).
__global__ void k_offgrid_interp(const float4* __restrict__ w, float4* __restrict__ wstar,
                                 const int2* __restrict__ first, const float* __restrict__ wts, int B, int by, int L2,
                                 int ndir, int Kx, int Ky) {
  const int k = blockIdx.y, blk = blockIdx.z;
  const int2 f0 = first[k];
  const float* cx = wts + (size_t)k * (Kx + Ky);
  const float* cy = cx + Kx;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L2; e += gridDim.x * blockDim.x) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = 0; i < Kx; ++i) {
      for (int j = 0; j < Ky; ++j) {
        const float c = cx[i] * cy[j];
        const float4 a = w[((size_t)blk * B + (size_t)(f0.x + i) * by + f0.y + j) * L2 + e];
        acc.x = fmaf(c, a.x, acc.x);
        acc.y = fmaf(c, a.y, acc.y);
        acc.z = fmaf(c, a.z, acc.z);
        acc.w = fmaf(c, a.w, acc.w);
      }
    }
    wstar[((size_t)blk * ndir + k) * L2 + e] = acc;
  }
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

}  // namespace
}  // namespace fbst

using namespace fbst;

struct fbst_offgrid_s {
  fbst_plan_s* plan;   // grid, stage 1, workspace and allocator (not owned)
  int ndir, Kx, Ky;
  fbst_plan_s shadow;  // stage-2 descriptor whose beams are the directions
  int2* first;         // [ndir] first grid index of the window along x and y
  float* wts;          // [ndir][Kx + Ky] spline weights along x, then y
  float2* wstar;       // [max_blocks][ndir][L]
};

static void free_offgrid(fbst_offgrid_s* o) {
  void* ptrs[] = {o->first, o->wts, o->wstar, o->shadow.XV, o->shadow.Aspec, o->shadow.pre_r, o->shadow.qspec_r,
                  o->shadow.post_r};
  for (void* q : ptrs) plan_free(o->plan, q);
}

static int offgrid_interp(fbst_offgrid_s* o, const float2* w, float2* wstar, int nb, cudaStream_t s) {
  const fbst_info& in = o->plan->info;
  const int L2 = in.L / 2;
  const dim3 grid((L2 + 255) / 256, o->ndir, nb);
  k_offgrid_interp<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(w), reinterpret_cast<float4*>(wstar),
                                        o->first, o->wts, in.B, o->plan->geom.by, L2, o->ndir, o->Kx, o->Ky);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

extern "C" {

int fbst_offgrid_create(fbst_offgrid_t* out, fbst_plan_t p, const double* directions, int ndir, int K, void* stream) {
  if (!out) return FBST_ERR_INVALID;
  *out = nullptr;
  if (!p || !directions || ndir < 1 || ndir > 65535 || K < 2 || K > kMaxWindow) return FBST_ERR_INVALID;
  if (p->nu_nf) return FBST_ERR_UNSUPPORTED;   // the off-grid generators use the grid positions
  const fbst_info& in = p->info;
  const fbst_geometry& g = p->geom;
  const bool ura = g.kind == FBST_URA;
  for (int k = 0; k < ndir; ++k) {
    const double u = directions[2 * k], v = directions[2 * k + 1];
    if (!std::isfinite(u) || !std::isfinite(v) || std::fabs(u) > 1.0 || std::fabs(v) > 1.0) return FBST_ERR_INVALID;
    if (!ura && v != 0.0) return FBST_ERR_INVALID;
  }
  int cur = -1;
  FBST_CUDA_TRY(cudaGetDevice(&cur));
  if (cur != p->device) return FBST_ERR_INVALID;
  const int Kx = std::min(K, g.bx), Ky = ura ? std::min(K, g.by) : 1;

  // Host: windows and spline weights (FP64), rounded to float once.
  std::vector<int2> first(ndir);
  std::vector<float> wts((size_t)ndir * (Kx + Ky));
  std::vector<double> dirs(directions, directions + 2 * (size_t)ndir);
  for (int k = 0; k < ndir; ++k) {
    int fx = 0, fy = 0;
    interp_terms(g.bx, g.by, ura, dirs[2 * k], dirs[2 * k + 1], Kx, Ky, &fx, &fy, &wts[(size_t)k * (Kx + Ky)]);
    first[k] = make_int2(fx, fy);
  }

  fbst_offgrid_s* o = new (std::nothrow) fbst_offgrid_s();
  if (!o) return FBST_ERR_OOM;
  std::memset(o, 0, sizeof(*o));
  o->plan = p;
  o->ndir = ndir;
  o->Kx = Kx;
  o->Ky = Ky;
  fbst_plan_s& sh = o->shadow;
  sh.info = in;
  sh.info.B = ndir;
  sh.info.stage2 = FBST_STAGE2_GS_IR1;
  sh.geom = g;
  sh.band = p->band;
  sh.device = p->device;
  sh.d_status = p->d_status;
  sh.tw32 = p->tw32;
  sh.tw64 = p->tw64;
  share_allocator(&sh, p);

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int maxb = p->band.max_blocks;
  double* dirs_dev = nullptr;
  int r = FBST_OK;
  do {
    if ((r = plan_alloc_n(p, &o->first, (size_t)ndir)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &o->wts, wts.size())) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &o->wstar, (size_t)maxb * ndir * in.L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &sh.XV, (size_t)ndir * 2 * in.P_gs)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &sh.Aspec, (size_t)ndir * in.P_gs)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &sh.pre_r, (size_t)in.L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &sh.qspec_r, (size_t)in.S_rec * in.P_rec)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &sh.post_r, (size_t)in.N)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &dirs_dev, dirs.size())) != FBST_OK) break;
    // Allocated in stream order on the plan's stream: make the blocks usable on `s`.
    if (cudaStreamSynchronize(p->mem_stream) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    if (cudaMemcpyAsync(o->first, first.data(), sizeof(int2) * ndir, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(o->wts, wts.data(), sizeof(float) * wts.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dirs_dev, dirs.data(), sizeof(double) * dirs.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      r = FBST_ERR_CUDA;
      break;
    }
    r = build_direction_operators(p, dirs_dev, ndir, sh.XV, sh.Aspec, sh.pre_r, sh.qspec_r, sh.post_r, s);
  } while (0);
  cudaStreamSynchronize(s);   // the host vectors above are read by the copies before they go
  plan_free(p, dirs_dev);
  if (r != FBST_OK) {
    free_offgrid(o);
    delete o;
    return r;
  }
  *out = o;
  return FBST_OK;
}

int fbst_offgrid_interpolate(fbst_offgrid_t o, const void* w, void* wstar, int nblk, void* stream) {
  if (!o || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!w || !wstar || !aligned16(w) || !aligned16(wstar)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = o->plan->info;
  for (int c0 = 0; c0 < nblk; c0 += 65535) {
    const int nb = std::min(65535, nblk - c0);
    FBST_TRY(offgrid_interp(o, static_cast<const float2*>(w) + (size_t)c0 * in.B * in.L,
                            static_cast<float2*>(wstar) + (size_t)c0 * o->ndir * in.L, nb, s));
  }
  return FBST_OK;
}

int fbst_offgrid_apply(fbst_offgrid_t o, const void* w, void* bstar, int nblk, void* stream) {
  if (!o || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!w || !bstar || !aligned16(w) || !aligned16(bstar)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = o->plan->info;
  const int maxb = std::min(o->plan->band.max_blocks, 65535);
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(offgrid_interp(o, static_cast<const float2*>(w) + (size_t)c0 * in.B * in.L, o->wstar, nb, s));
    FBST_TRY(launch_stage2_gs(&o->shadow, o->wstar, static_cast<float2*>(bstar) + (size_t)c0 * o->ndir * in.N, nb, s));
  }
  return FBST_OK;
}

int fbst_offgrid_execute(fbst_offgrid_t o, const void* y, void* bstar, int nblk, void* stream) {
  if (!o || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!y || !bstar || !aligned16(y) || !aligned16(bstar)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fbst_plan_s* p = o->plan;
  const fbst_info& in = p->info;
  const int maxb = std::min(p->band.max_blocks, 65535);
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    FBST_TRY(launch_czt_time(p, static_cast<const float2*>(y) + (size_t)c0 * in.M * in.N, p->ws_yhat, nb, s));
    FBST_TRY(launch_czt_space(p, p->ws_yhat, p->ws_w, nb, s));
    FBST_TRY(offgrid_interp(o, p->ws_w, o->wstar, nb, s));
    FBST_TRY(launch_stage2_gs(&o->shadow, o->wstar, static_cast<float2*>(bstar) + (size_t)c0 * o->ndir * in.N, nb, s));
  }
  return FBST_OK;
}

int fbst_offgrid_destroy(fbst_offgrid_t o) {
  if (!o) return FBST_OK;
  free_offgrid(o);
  delete o;
  return FBST_OK;
}

}  // extern "C"
