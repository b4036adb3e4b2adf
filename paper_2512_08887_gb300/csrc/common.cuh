// Shared definitions of the FBST CUDA library: complex helpers, the plan object and error macros.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fbst.h"

namespace fbst {

// ---------------------------------------------------------------------------------------------
// Complex arithmetic on float2 / double2 (x = real, y = imaginary).
// ---------------------------------------------------------------------------------------------
template <typename R> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };

template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
  return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
  return V{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
template <typename V> __host__ __device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) {
  return V{a.x * s, a.y * s};
}

// Largest FFT size of any table or kernel, and the size of the shared twiddle tables (the ladder:
// exp(-2*pi*i*k/M) for k < M/2 at index M/2 - 1 + k, every power of two M <= kMaxFFT, built in
// FP64 at plan time).
constexpr int kMaxFFT = 4096;
constexpr int kTwiddleSize = 4096;

}  // namespace fbst

// ---------------------------------------------------------------------------------------------
// Jobs: one plan's share of a stage launch. A launch takes up to kMaxJobs jobs of the same
// transform size and shape (passed by value as a __grid_constant__ parameter), flattens their
// work items and splits them evenly over the resident CTAs. A single-plan call is a one-job launch;
// a batch of uneven arrays groups its plans' jobs by transform size.
// ---------------------------------------------------------------------------------------------
namespace fbst {
constexpr int kMaxJobs = 32;

struct time_job {      // temporal chirp-z of one plan over nblk blocks
  const float2* y;
  float2* yhat;
  const float2* pre;
  const float2* gspec;
  const float2* post;
  int M, N, L, S, nblk;
  long long first;     // first flattened work item of this job
  long long ys_m, ys_b;  // elements between the rows of two sensors / the starts of two blocks in y
                         // (N and M*N for [nblk][M][N]; T and the hop for a continuous record [M][T])
};

struct space_job {     // spatial chirp-z (linear array) of one plan over nblk blocks
  const float2* yhat;
  float2* w;
  const float2* pre;
  const float2* kspec;
  const float2* post;
  int M, B, L, nblk;
  long long first;
  unsigned* wmax;      // null, or [nblk]: atomic max of |re|, |im| of each block's w (float bits)
};

struct gs_job {        // Gohberg-Semencul stage 2 + reconstruction of one plan over nblk blocks
  const float2* w;
  float2* bhat;
  const float2* XV;
  const float2* Aspec;
  const float2* pre_r;
  const float2* qspec;
  const float2* post_r;
  int B, L, N, nblk;
  long long first;
};

template <typename J>
struct job_list {
  J job[kMaxJobs];
  int n;
  long long total;     // total work items over all jobs
};

// Launch shape of a Stockham kernel: elements per thread (the radix) and transforms per CTA.
struct fft_shape {
  int E;
  int G;
};
}  // namespace fbst

// ---------------------------------------------------------------------------------------------
// The plan. All pointers are device memory owned by the plan unless stated otherwise.
// ---------------------------------------------------------------------------------------------
struct fbst_axis_tables {
  int Ma, Ba, P;       // elements along the axis, beams along the axis, Bluestein FFT size
  float2* pre;         // [L][Ma]   chirp premultiply (includes the -kappa*m steering offset)
  float2* kspec;       // [L][P]    FFT of the Bluestein kernel, scaled by 1/P
  float2* post;        // [L][Ba]   chirp postmultiply
};

namespace fbst {
struct mem_registry;   // every live device block of a plan with its size (api.cu)
}

struct fbst_plan_s {
  fbst_info info;
  fbst_geometry geom;
  fbst_band band;
  int device;

  // Device memory of the plan (tables, workspace, staging, temporaries, nulling objects) comes
  // from the caller's allocator, or from cudaMallocAsync / cudaFreeAsync when none is given, and is
  // always allocated and freed in stream order on mem_stream (the stream given to fbst_plan).
  fbst_alloc_fn alloc_fn;
  fbst_free_fn free_fn;
  void* alloc_ctx;
  cudaStream_t mem_stream;
  fbst::mem_registry* mem;

  float2* tw32;        // [kTwiddleSize] twiddle ladder (see kTwiddleSize) rounded to float
  double2* tw64;       // same in double (plan-time FFTs)

  // Stage 1a: temporal chirp-z (N snapshots -> L frequencies), S_time output splits.
  float2* pre_t;       // [N]
  float2* gspec_t;     // [S_time][P_time], scaled by 1/P_time
  float2* post_t;      // [L]

  // Stage 1b of a non-uniform linear array (Sec. IX): element x positions and the type-1 NUFFT
  // tables (nu_nf = 0 for arrays on the grid, which use the chirp-z tables below).
  int nu_nf;           // oversampled grid size (power of two >= 2B), = info.P_space_x
  int nu_w;            // spreading width in grid points
  double* pos;         // [M] element positions along x, half wavelengths
  int* nu_j0;          // [L][M] first grid point each element reaches
  float* nu_dg;        // [L][M] its grid coordinate minus that point, in (nu_w/2 - 1, nu_w/2]
  float* nu_deconv;    // [bx] 1 / kernel Fourier transform at the beam's mode (and / nu_nf scale)
  // A rectangular array off the grid: the y axis of the two-dimensional NUFFT (nu_nfy = 0 for a
  // linear array); nu_j0 / nu_dg / nu_deconv above then hold the x axis.
  int nu_nfy;          // oversampled grid size along y (power of two >= 2 by), = info.P_space_y
  double* pos_y;       // [M] element positions along y, half wavelengths
  int* nu_j0y;         // [L][M]
  float* nu_dgy;       // [L][M]
  float* nu_deconv_y;  // [by]

  // Stage 1b: spatial chirp-z per frequency; axis 0 = x (all arrays), axis 1 = y (rectangular).
  fbst_axis_tables ax[2];
  int n_axes;
  int same_axes;       // 1 if the y axis reuses axis 0's tables

  // Stage 2, Gohberg-Semencul: spectra of x_b and of Z J conj(x_b), both / (sqrt(x_0) * P_gs),
  // stored together per beam: XV[b][0][k] = X_b[k], XV[b][1][k] = V_b[k].
  float2* XV;          // [B][2][P_gs]
  // Spectrum of the circulant embedding of A_b (size P_gs), / P_gs, for the refinement step.
  float2* Aspec;       // [B][P_gs] (GS_IR1 only)
  // Reconstruction chirp-z F_u (L coefficients -> N samples), S_rec input splits.
  float2* pre_r;       // [S_rec][L/S_rec]
  float2* qspec_r;     // [S_rec][P_rec], scaled by 1/P_rec
  float2* post_r;      // [N]

  // Stage 2, dense: G_b = F_u A_b^{-1}.
  float2* G;           // [B][N][L] complex64 (DENSE_FP32)
  void* Gtc;           // tensor-core operand (split-BF16 or TF32 layout), see dense_tc.cu
  size_t Gtc_bytes;
  int* tc_gexp;        // [B] FP16 split: exponent of each beam's scale of G
  unsigned* tc_wmax;   // [max_blocks] FP16 split: largest |re|, |im| of each block of w (float bits)
  bool tc_wmax_stage1; // FP16 split on a linear grid array: the spatial chirp-z writes tc_wmax

  double2* x64;        // [B][L] first column of A_b^{-1} (FP64), kept for inspection

  // Per-call workspace, max_blocks blocks.
  float2* ws_yhat;     // [max_blocks][L][M]
  float2* ws_w;        // [max_blocks][B][L]
  void* ws_tc;         // tensor-core right-hand-side operand (dense TC variants)
  size_t ws_tc_bytes;

  // Host-buffer staging (fbst_execute_host), allocated on first use, with the two copy streams
  // and the events of its pipeline (copies in / out overlapped with the kernels).
  float2* stage_y;     // [max_blocks][M][N]
  float2* stage_bhat;  // [max_blocks][B][N]
  cudaStream_t copy_in, copy_out;
  cudaEvent_t pipe_ev[12];

  float2* stream_bhat; // [max_blocks][B][N] block outputs of fbst_execute_stream (first use)

  int* d_status;       // device status word (FP64 plan kernels report here)
  // Limit of one pipeline wait of the tensor-core stage-2 kernels, ns (0 = the default, 1 s);
  // a wait that runs out makes the kernel record FBST_ERR_TIMEOUT, drain its copies and return.
  unsigned long long wait_ns;

  // Stage trace (fbst_trace_stages): 4 timing events per traced fbst_execute call in a ring of
  // trace_cap calls; trace_next counts the calls traced, trace_count those not yet read.
  cudaEvent_t* trace_ev;
  int trace_cap, trace_next, trace_count;

  // Launch shapes of the temporal and spatial chirp-z kernels ({0, 0} = built-in default;
  // fbst_autotune / fbst_set_shapes change them).
  fbst::fft_shape shape_time;
  fbst::fft_shape shape_space;
};

#define FBST_CUDA_TRY(expr)                                  \
  do {                                                       \
    cudaError_t fbst_e_ = (expr);                            \
    if (fbst_e_ != cudaSuccess) {                            \
      fbst::set_last_cuda_error(fbst_e_, #expr, __FILE__, __LINE__); \
      return FBST_ERR_CUDA;                                  \
    }                                                        \
  } while (0)

namespace fbst {
void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void set_last_error_message(const char* msg);

// Plan memory (api.cu). plan_alloc returns FBST_ERR_OOM when the allocator has no memory (and
// FBST_ERR_INVALID for a block that is not 16-byte aligned); bytes = 0 gives a null pointer.
// plan_free returns a block of this plan's registry (null and unknown pointers are ignored).
int plan_alloc(fbst_plan_s* p, size_t bytes, void** out);
void plan_free(fbst_plan_s* p, void* ptr);
template <typename T>
int plan_alloc_n(fbst_plan_s* p, T** out, size_t count) {
  void* q = nullptr;
  const int r = plan_alloc(p, count * sizeof(T), &q);
  *out = static_cast<T*>(q);
  return r;
}
// dst uses src's allocator and registry (a descriptor that shares the plan's memory accounting).
inline void share_allocator(fbst_plan_s* dst, const fbst_plan_s* src) {
  dst->alloc_fn = src->alloc_fn;
  dst->free_fn = src->free_fn;
  dst->alloc_ctx = src->alloc_ctx;
  dst->mem_stream = src->mem_stream;
  dst->mem = src->mem;
}

// Kernel launchers (each returns an fbst_status). All run on `s`.
int launch_czt_time(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk, cudaStream_t s);
// The temporal chirp-z of nblk blocks read in place from a continuous record [M][T] (sample
// fastest): block k is samples [k*hop, k*hop + N) of every sensor's row.
int launch_czt_time_record(const fbst_plan_s* p, const float2* record, long long T, int hop, float2* yhat, int nblk,
                           cudaStream_t s);
int launch_czt_space(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s);
// The same, and when p->tc_wmax_stage1 also the block maxima of w into p->tc_wmax + blk0 (blocks
// blk0 .. blk0 + nblk - 1 of the chunk that stage 2 will take).
int launch_czt_space_scaled(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, int blk0,
                            cudaStream_t s);
int launch_stage2_gs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s);

// Multi-job launchers: every job of `jl` shares the transform size P (and for stage 2 the
// reconstruction size/splits and the refinement flag).
int launch_time_jobs(const job_list<time_job>& jl, int P, fft_shape shape, int max_Lh, const float2* tw,
                     cudaStream_t s);
int launch_space_jobs(const job_list<space_job>& jl, int P, fft_shape shape, int max_B, const float2* tw,
                      cudaStream_t s);
int launch_gs_jobs(const job_list<gs_job>& jl, int PG, int PR, int SR, bool IR, int max_L, const float2* tw,
                   cudaStream_t s);
// Job of one plan for nblk blocks (first = 0), and the shape the plan uses for it.
time_job make_time_job(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk);
space_job make_space_job(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk);
gs_job make_gs_job(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk);
fft_shape time_shape(const fbst_plan_s* p);
fft_shape space_shape(const fbst_plan_s* p);
// Shapes that have a compiled kernel for transform size P (fills up to `cap` entries).
int time_shapes(int P, fft_shape* out, int cap);
int space_shapes(int P, fft_shape* out, int cap);
// Work items of a job (for the flattened ranges) given the launch shape.
long long time_items(const time_job& j, fft_shape sh, int P);
long long space_items(const space_job& j, fft_shape sh, int P);
int launch_stage2_dense_fp32(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s);
// The same kernel with one right-hand side per block shared by every beam (w [nblk][L]) when
// shared_rhs is set.
int launch_dense_fp32_rhs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, bool shared_rhs,
                          cudaStream_t s);
// scales_ready: tc_wmax already holds the block maxima of this w (written by the spatial chirp-z).
int launch_stage2_dense_tc(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s,
                           bool scales_ready = false);
// The TF32x3 operator for beams [b0, b0 + nbeam) only (FBST_ERR_UNSUPPORTED for other variants).
int launch_stage2_dense_tc_beams(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, int b0, int nbeam,
                                 cudaStream_t s);
// The TF32x3 operator of every beam applied to one right-hand side per block, w [nblk][L] (the
// same for all beams); bhat [nblk][B][N].
int launch_dense_tc_shared_rhs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s);
// FP16-split tensor-core stage 2: the block maxima of w in tc_wmax, from w itself (no-op for the
// other variants); stage 2 calls it unless the spatial chirp-z has written them, a caller that runs
// stage 2 by beam ranges calls it once before the ranges.
int prepare_dense_tc_scales(const fbst_plan_s* p, const float2* w, int nblk, cudaStream_t s);
int stage2_launches(const fbst_plan_s* p, bool w_from_stage1);
// Stage 2 of the plan's variant on w [nb][B][L] -> bhat [nb][B][N] (nb <= max_blocks).
// w_from_stage1: w was written by launch_czt_space_scaled with the plan's tc_wmax in this call.
int run_stage2(const fbst_plan_s* p, const float2* w, float2* bhat, int nb, cudaStream_t s,
               bool w_from_stage1 = false);

// Plan-time builders (plan.cu / dense_tc.cu).
int build_plan_tables(fbst_plan_s* p, cudaStream_t s);
int build_dense_tc_operand(fbst_plan_s* p, cudaStream_t s);
// FP64 first columns x of A^{-1} for `count` arbitrary directions (dirs_dev: device [count][2]);
// the status word reports a generator that is not positive definite (plan.cu).
int build_direction_x(fbst_plan_s* p, const double* dirs_dev, int count, double2* x, cudaStream_t s);
// Non-uniform stage 1b: kernel shape for a width of W grid points, and the deconvolution factors
// of the plan's beams (plan.cu).
double nufft_beta(int W);
int nufft_deconv(fbst_plan_s* p, cudaStream_t s);
// Stage-2 operators of `count` arbitrary directions (dirs_dev: device [count][2] direction cosines
// (u, v)): Gohberg-Semencul spectra XV [count][2][P_gs], circulant spectra Aspec [count][P_gs] (may
// be null) and the reconstruction tables of the plan's F_u, all from FP64 (plan.cu).
int build_direction_operators(fbst_plan_s* p, const double* dirs_dev, int count, float2* XV, float2* Aspec,
                              float2* pre_r, float2* qspec_r, float2* post_r, cudaStream_t s);
// In-place FP64 FFT of `rows` contiguous rows of size P (dir -1 forward, +1 unnormalised inverse).
int fft64_rows(double2* data, int rows, int P, const double2* tw, int dir, cudaStream_t s);
// Toeplitz generators a_b(d) of the plan's beams in FP64 (Sec. V), [B][L] (plan.cu).
int plan_toeplitz_generators(fbst_plan_s* p, double2* gen, cudaStream_t s);
// x = A^{-1} e_0 for `count` generators [count][L] by the Levinson recursion (plan.cu) or by the
// method of enum fbst_generator_solver (superfast.cu); a non-positive pivot records
// FBST_ERR_NUMERIC in the plan's status word.
int launch_levinson(const double2* gen, double2* x, int count, int L, int* status, cudaStream_t s);
int solve_generators(fbst_plan_s* p, const double2* gen, double2* x, int count, int method, cudaStream_t s);
}  // namespace fbst
