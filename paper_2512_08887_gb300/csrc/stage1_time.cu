// Temporal chirp-z of stage 1 (Sec. IV, the sum over snapshots):
//   yhat[m, ell] = sum_n y[m, n] exp(-2*pi*i*eps*ell'*n/L),   ell' = ell + 1 - L/2,
// by Bluestein with the output split into S halves that share one forward transform of size P:
// premultiply by the chirp, FFT, multiply by the kernel spectrum of half h, inverse FFT, post-
// multiply (tables from plan.cu). Layout y [blk][M][N] (or blocks read in place from a continuous
// record [M][T], the job's strides) -> yhat [blk][L][M]: a work item is G
// consecutive elements of one block (one Stockham group each); the transpose goes through shared
// memory and leaves as G-element runs (32 bytes for G = 4) so global stores fill whole sectors.
//
// The grid holds exactly the CTAs that fit on the GPU (occupancy x SMs); CTA c takes the
// contiguous range [c*I/Gd, (c+1)*I/Gd) of the I work items of all jobs of the launch.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "launch_util.cuh"

namespace fbst {

// HALF: every job has N = L/S = P/2, so snapshot n < N and output i < L/S are exactly the slots
// r < E/2 of each thread (the zero upper half of the input and the unused upper half of each
// output are known at compile time).
template <int P, int E, int G, bool HALF>
__global__ void __launch_bounds__(G * (P / E))
k_czt_time(const __grid_constant__ job_list<time_job> jl, const float2* __restrict__ tw) {
  constexpr int T = P / E;
  constexpr int SB = fft_smem_elems<float2>(P);
  static_assert(T <= 32 || G <= 15, "named barriers 1..15, one per transform group");
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  float2* fbuf = sm + g * SB;
  float2* tile = sm + G * SB;  // [Lh][G + 1] (padded row: conflict-free column writes)
  long long it0, it1;
  my_range(jl.total, &it0, &it1);
  int j = 0;
  for (long long it = it0; it < it1; ++it) {
    while (j + 1 < jl.n && jl.job[j + 1].first <= it) ++j;
    const time_job& J = jl.job[j];
    const int M = J.M, N = J.N, L = J.L, S = J.S, Lh = L / S;
    const int ntile = (M + G - 1) / G;
    const long long li = it - J.first;
    const int blk = (int)(li / ntile), m0 = (int)(li % ntile) * G;
    const int m = m0 + g;
    const float2* yrow = J.y + (size_t)blk * J.ys_b + (size_t)(m < M ? m : M - 1) * J.ys_m;
    float2 v[1][E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int n = t + T * r;
      v[0][r] = ((HALF ? r < E / 2 : n < N) && m < M) ? cmul(yrow[n], J.pre[n]) : make_float2(0.f, 0.f);
    }
    block_fft<P, E, 1, -1>(v, fbuf, tw, t, 1 + g);
    for (int h = 0; h < S; ++h) {
      float2 u[1][E];
#pragma unroll
      for (int r = 0; r < E; ++r) u[0][r] = cmul(v[0][r], J.gspec[h * P + t + T * r]);
      block_fft<P, E, 1, +1>(u, fbuf, tw, t, 1 + g);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = t + T * r;
        if (HALF ? r < E / 2 : i < Lh) tile[i * (G + 1) + g] = cmul(u[0][r], J.post[h * Lh + i]);
      }
      __syncthreads();
      float2* out = J.yhat + ((size_t)blk * L + (size_t)h * Lh) * M + m0;
      for (int idx = threadIdx.x; idx < Lh * G; idx += blockDim.x) {
        const int i = idx / G, gg = idx % G;
        if (m0 + gg < M) out[(size_t)i * M + gg] = tile[i * (G + 1) + gg];
      }
      __syncthreads();
    }
  }
}

template <int P, int E, int G, bool HALF>
static int run_time(const job_list<time_job>& jl, int max_Lh, const float2* tw, cudaStream_t s) {
  constexpr int T = P / E;
  const size_t smem = sizeof(float2) * ((size_t)G * fft_smem_elems<float2>(P) + (size_t)max_Lh * (G + 1));
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_czt_time<P, E, G, HALF>));
  const int grid = grid_for_items(jl.total, resident_ctas(k_czt_time<P, E, G, HALF>, G * T, smem));
  k_czt_time<P, E, G, HALF><<<grid, G * T, smem, s>>>(jl, tw);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// Every job of the list has N = L/S = P/2 (the compile-time half-size form applies).
static bool time_jobs_half(const job_list<time_job>& jl, int P) {
  for (int i = 0; i < jl.n; ++i)
    if (2 * jl.job[i].N != P || 2 * (jl.job[i].L / jl.job[i].S) != P) return false;
  return true;
}

// Compiled shapes (P, E, G): G*P/E <= 512 threads. The first entry of each P is its default.
#define FBST_TIME_SHAPES(X)                                                                          \
  X(16, 8, 16) X(32, 8, 16) X(64, 8, 16) X(64, 8, 8) X(128, 8, 8) X(128, 8, 4) X(128, 16, 8)           \
  X(256, 8, 8) X(256, 8, 4) X(256, 8, 2) X(256, 16, 8) X(256, 16, 4) X(512, 16, 8) X(512, 8, 4)         \
  X(512, 8, 2) X(512, 8, 8) X(512, 16, 4) X(512, 16, 2) X(1024, 16, 4) X(1024, 8, 4) X(1024, 8, 2)    \
  X(1024, 16, 8) X(1024, 16, 2) X(2048, 16, 4) X(2048, 16, 2) X(2048, 8, 2) X(4096, 16, 2)

int launch_time_jobs(const job_list<time_job>& jl, int P, fft_shape sh, int max_Lh, const float2* tw,
                     cudaStream_t s) {
  if (jl.total <= 0) return FBST_OK;
  // The half-size form is compiled for the radix-16 shapes (the defaults of the large transforms).
  const bool half = time_jobs_half(jl, P);
#define FBST_X(p, e, g)                                                                               \
  if (P == p && sh.E == e && sh.G == g)                                                               \
    return (half && e == 16) ? run_time<p, e, g, (e == 16)>(jl, max_Lh, tw, s)                        \
                             : run_time<p, e, g, false>(jl, max_Lh, tw, s);
  FBST_TIME_SHAPES(FBST_X)
#undef FBST_X
  return FBST_ERR_UNSUPPORTED;
}

int time_shapes(int P, fft_shape* out, int cap) {
  int n = 0;
#define FBST_X(p, e, g) \
  if (P == p && n < cap) out[n++] = fft_shape{e, g};
  FBST_TIME_SHAPES(FBST_X)
#undef FBST_X
  return n;
}

fft_shape time_shape(const fbst_plan_s* p) {
  if (p->shape_time.E) return p->shape_time;
  fft_shape d{0, 0};
  time_shapes(p->info.P_time, &d, 1);
  return d;
}

long long time_items(const time_job& j, fft_shape sh, int) {
  return (long long)((j.M + sh.G - 1) / sh.G) * j.nblk;
}

time_job make_time_job(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk) {
  const fbst_info& in = p->info;
  return time_job{y, yhat, p->pre_t, p->gspec_t, p->post_t, in.M, in.N, in.L, in.S_time, nblk, 0,
                  (long long)in.N, (long long)in.M * in.N};
}

int launch_czt_time_record(const fbst_plan_s* p, const float2* record, long long T, int hop, float2* yhat, int nblk,
                           cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  job_list<time_job> jl;
  jl.n = 1;
  jl.job[0] = make_time_job(p, record, yhat, nblk);
  jl.job[0].ys_m = T;
  jl.job[0].ys_b = hop;
  const fft_shape sh = time_shape(p);
  jl.total = time_items(jl.job[0], sh, p->info.P_time);
  return launch_time_jobs(jl, p->info.P_time, sh, p->info.L / p->info.S_time, p->tw32, s);
}

int launch_czt_time(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk, cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  job_list<time_job> jl;
  jl.n = 1;
  jl.job[0] = make_time_job(p, y, yhat, nblk);
  const fft_shape sh = time_shape(p);
  jl.total = time_items(jl.job[0], sh, p->info.P_time);
  return launch_time_jobs(jl, p->info.P_time, sh, p->info.L / p->info.S_time, p->tw32, s);
}

}  // namespace fbst
