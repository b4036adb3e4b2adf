// Spatial chirp-z of stage 1 (Sec. IV, the sum over elements; App. B for rectangular arrays):
//   w[b, ell] = sum_m yhat[m, ell] exp(2*pi*i*kappa_ell*(u_b.p_m)),  kappa_ell = rho*(1/fb + eps*ell'/L),
// one Bluestein chirp-z per frequency with a frequency-dependent chirp rate (tables from plan.cu).
// Layout yhat [blk][L][M] -> w [blk][B][L]: a work item is G consecutive frequencies of one block;
// the transpose goes through shared memory and leaves as G-frequency runs (32-byte sectors).
// Work items are tile-major, so a CTA's contiguous range mostly stays on one frequency tile and
// keeps that tile's chirps and kernel spectrum in registers.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "launch_util.cuh"

namespace fbst {

// At least 512 threads per SM (128 registers a thread): the kernel lives on latency hiding.
// HALF: every job has M = B = P/2, so element i < M and beam b < B are exactly the slots r < E/2
// of each thread; the zero upper half of the input and the unused upper half of the output are
// then known at compile time (the first forward pass and the last inverse pass lose that work).
template <int P, int E, int G, bool HALF>
__global__ void __launch_bounds__(G * (P / E), G * (P / E) >= 512 ? 1 : 512 / (G * (P / E)))
k_czt_space_ula(const __grid_constant__ job_list<space_job> jl, const float2* __restrict__ tw, int max_B) {
  constexpr int T = P / E;
  constexpr int SB = fft_smem_elems<float2>(P);
  static_assert(T <= 32 || G <= 15, "named barriers 1..15, one per transform group");
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  float2* fbuf = sm + g * SB;
  float2* tile = sm + G * SB;  // [B][G + 1] (padded row: conflict-free column writes)
  // Block maxima of w for the FP16-split stage 2 (only for a launch of one job that asks for them):
  // this CTA's per-block words after the tile, zeroed here, combined into the job's at the end.
  unsigned* wmax_s = nullptr;
  if (jl.n == 1 && jl.job[0].wmax) {
    wmax_s = reinterpret_cast<unsigned*>(tile + (size_t)max_B * (G + 1));
    for (int i = threadIdx.x; i < jl.job[0].nblk; i += blockDim.x) wmax_s[i] = 0u;
    __syncthreads();
  }
  long long it0, it1;
  my_range(jl.total, &it0, &it1);
  int j = 0, cur_j = -1, cur_lt = -1;
  float2 pr[E <= 8 ? E : 1], ks[E <= 8 ? E : 1], po[E <= 8 ? E : 1];
  for (long long it = it0; it < it1; ++it) {
    while (j + 1 < jl.n && jl.job[j + 1].first <= it) ++j;
    const space_job& J = jl.job[j];
    const int M = J.M, B = J.B, L = J.L, nblk = J.nblk;
    const long long li = it - J.first;
    const int lt = (int)(li / nblk), blk = (int)(li % nblk);
    const int ell0 = lt * G;
    const int ell = ell0 + g;
    const int ellc = ell < L ? ell : L - 1;
    const float2* row = J.yhat + ((size_t)blk * L + ellc) * M;
    float2 v[1][E];
    if constexpr (E <= 8) {
      // Radix 8: a frequency tile's chirp / spectrum rows stay in registers across the blocks
      // that share them.
      if (lt != cur_lt || j != cur_j) {
        cur_lt = lt;
        cur_j = j;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int i = t + T * r;
          pr[r] = (HALF ? r < E / 2 : i < M) ? J.pre[(size_t)ellc * M + i] : make_float2(0.f, 0.f);
          ks[r] = J.kspec[(size_t)ellc * P + i];
          po[r] = (HALF ? r < E / 2 : i < B) ? J.post[(size_t)ellc * B + i] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = t + T * r;
        v[0][r] = (HALF ? r < E / 2 : i < M) ? cmul(row[i], pr[r]) : make_float2(0.f, 0.f);
      }
      block_fft<P, E, 1, -1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
      for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], ks[r]);
      block_fft<P, E, 1, +1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int b = t + T * r;
        if (HALF ? r < E / 2 : b < B) tile[b * (G + 1) + g] = cmul(v[0][r], po[r]);
      }
    } else {
      // Radix 16 has no registers to spare: the rows are read from L1 where they are used.
      const float2* pre = J.pre + (size_t)ellc * M;
      const float2* kspec = J.kspec + (size_t)ellc * P;
      const float2* post = J.post + (size_t)ellc * B;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = t + T * r;
        v[0][r] = (HALF ? r < E / 2 : i < M) ? cmul(row[i], pre[i]) : make_float2(0.f, 0.f);
      }
      block_fft<P, E, 1, -1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
      for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], kspec[t + T * r]);
      block_fft<P, E, 1, +1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int b = t + T * r;
        if (HALF ? r < E / 2 : b < B) tile[b * (G + 1) + g] = cmul(v[0][r], post[b]);
      }
    }
    __syncthreads();
    float2* out = J.w + (size_t)blk * B * L + ell0;
    float wm = 0.f;
    for (int idx = threadIdx.x; idx < B * G; idx += blockDim.x) {
      const int b = idx / G, gg = idx % G;
      if (ell0 + gg < L) {
        const float2 o = tile[b * (G + 1) + gg];
        out[(size_t)b * L + gg] = o;
        wm = fmaxf(wm, fmaxf(fabsf(o.x), fabsf(o.y)));
      }
    }
    if (wmax_s) {
      // The block's largest |re|, |im| (the scale of the FP16-split stage 2): a warp maximum into
      // this CTA's per-block word (non-negative floats order like their bit patterns).
      for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
      if ((threadIdx.x & 31) == 0) atomicMax(wmax_s + blk, __float_as_uint(wm));
    }
    __syncthreads();
  }
  if (wmax_s) {
    // One global atomic per block this CTA touched (the CTA's items are a contiguous range).
    for (int i = threadIdx.x; i < jl.job[0].nblk; i += blockDim.x)
      if (wmax_s[i]) atomicMax(jl.job[0].wmax + i, wmax_s[i]);
  }
}

template <int P, int E, int G, bool HALF>
static int run_space(const job_list<space_job>& jl, int max_B, const float2* tw, cudaStream_t s) {
  constexpr int T = P / E;
  const size_t wm = (jl.n == 1 && jl.job[0].wmax) ? sizeof(unsigned) * (size_t)jl.job[0].nblk : 0;
  const size_t smem = sizeof(float2) * ((size_t)G * fft_smem_elems<float2>(P) + (size_t)max_B * (G + 1)) + wm;
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_czt_space_ula<P, E, G, HALF>));
  const int grid = grid_for_items(jl.total, resident_ctas(k_czt_space_ula<P, E, G, HALF>, G * T, smem));
  k_czt_space_ula<P, E, G, HALF><<<grid, G * T, smem, s>>>(jl, tw, max_B);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// Every job of the list has M = B = P/2 (the compile-time half-size form applies).
static bool space_jobs_half(const job_list<space_job>& jl, int P) {
  for (int i = 0; i < jl.n; ++i)
    if (2 * jl.job[i].M != P || 2 * jl.job[i].B != P) return false;
  return true;
}

// Compiled shapes (P, E, G); the first entry of each P is its default.
#define FBST_SPACE_SHAPES(X)                                                                         \
  X(16, 8, 16) X(32, 8, 16) X(64, 8, 16) X(64, 8, 8) X(128, 8, 8) X(128, 8, 4) X(128, 16, 8)           \
  X(256, 8, 8) X(256, 8, 4) X(256, 8, 2) X(256, 16, 8) X(256, 16, 4) X(512, 8, 4) X(512, 8, 2)         \
  X(512, 8, 8) X(512, 16, 4) X(512, 16, 8) X(512, 16, 2) X(1024, 8, 4) X(1024, 8, 2) X(1024, 16, 4)    \
  X(1024, 16, 8) X(1024, 16, 2) X(2048, 16, 4) X(2048, 16, 2) X(2048, 8, 2) X(4096, 16, 2)

int launch_space_jobs(const job_list<space_job>& jl, int P, fft_shape sh, int max_B, const float2* tw,
                      cudaStream_t s) {
  if (jl.total <= 0) return FBST_OK;
  // The half-size form is compiled for the radix-16 shapes (the defaults of the large transforms).
  const bool half = space_jobs_half(jl, P);
#define FBST_X(p, e, g)                                                                               \
  if (P == p && sh.E == e && sh.G == g)                                                               \
    return (half && e == 16) ? run_space<p, e, g, (e == 16)>(jl, max_B, tw, s)                        \
                             : run_space<p, e, g, false>(jl, max_B, tw, s);
  FBST_SPACE_SHAPES(FBST_X)
#undef FBST_X
  return FBST_ERR_UNSUPPORTED;
}

int space_shapes(int P, fft_shape* out, int cap) {
  int n = 0;
#define FBST_X(p, e, g) \
  if (P == p && n < cap) out[n++] = fft_shape{e, g};
  FBST_SPACE_SHAPES(FBST_X)
#undef FBST_X
  return n;
}

fft_shape space_shape(const fbst_plan_s* p) {
  if (p->shape_space.E) return p->shape_space;
  fft_shape d{0, 0};
  space_shapes(p->info.P_space_x, &d, 1);
  return d;
}

long long space_items(const space_job& j, fft_shape sh, int) {
  return (long long)((j.L + sh.G - 1) / sh.G) * j.nblk;
}

space_job make_space_job(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk) {
  const fbst_axis_tables& ax = p->ax[0];
  return space_job{yhat, w, ax.pre, ax.kspec, ax.post, ax.Ma, ax.Ba, p->info.L, nblk, 0, nullptr};
}

// ---------------------------------------------------------------------------------------------
// Rectangular array (App. B): for each frequency, a chirp-z along y (my -> by) for every row kx,
// then along x (mx -> bx) for every beam column c, both in shared memory. Work item = (tile of
// TL consecutive frequencies, block). Both axes use size-P transforms.
// ---------------------------------------------------------------------------------------------
template <int P> struct ura_e { static constexpr int value = P >= 2048 ? 16 : (P >= 8 ? 8 : 2); };

template <int P, int TL, int NTH>
__global__ void __launch_bounds__(NTH)
k_czt_space_ura(const float2* __restrict__ yhat, float2* __restrict__ w, fbst_axis_tables axx,
                fbst_axis_tables axy, const float2* __restrict__ tw, int L, int nblk) {
  constexpr int E = ura_e<P>::value;
  constexpr int T = P / E;
  constexpr int G = NTH / T;  // concurrent transforms
  constexpr int SB = fft_smem_elems<float2>(P);
  static_assert(T <= 32 || G <= 15, "named barriers 1..15, one per transform group");
  extern __shared__ float2 sm[];
  const int mx = axx.Ma, bx = axx.Ba, my = axy.Ma, by = axy.Ba;
  const int M = mx * my, B = bx * by;
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  static_assert(TL == 4, "the tile swizzle permutes the 4 frequencies of a slot");
  float2* fbuf = sm + g * SB;
  // Z [mx][zs] and the output tile [bx][ts] are swizzled so that neither the row-wise nor the
  // column-wise accesses of a half-warp (two transform groups of 8) share a bank: Z column c of
  // row kx sits at c ^ (kx & 7) with rows round8(by) + 8 apart; the frequency j of output
  // (a, c) sits at c*TL + (j ^ (a & 3)) with rows by*TL + 2 apart. Both only permute within
  // aligned groups, so every index stays inside its row.
  const int zs = ((by + 7) & ~7) + 8, ts = by * TL + 2;
  float2* Z = sm + G * SB;
  float2* tile = Z + mx * zs;
  const int ntile = (L + TL - 1) / TL;
  long long it0, it1;
  my_range((long long)ntile * nblk, &it0, &it1);
  for (long long it = it0; it < it1; ++it) {
    const int lt = (int)(it / nblk), blk = (int)(it % nblk);
    const int ell0 = lt * TL;
    for (int j = 0; j < TL; ++j) {
      const int ell = min(ell0 + j, L - 1);
      const float2* src = yhat + ((size_t)blk * L + ell) * M;
      for (int kx0 = 0; kx0 < mx; kx0 += G) {
        const int kx = kx0 + g;
        const bool act = kx < mx;
        float2 v[1][E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int ky = t + T * r;
          v[0][r] = (act && ky < my) ? cmul(src[kx * my + ky], axy.pre[(size_t)ell * my + ky]) : make_float2(0.f, 0.f);
        }
        block_fft<P, E, 1, -1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
        for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], axy.kspec[(size_t)ell * P + t + T * r]);
        block_fft<P, E, 1, +1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int c = t + T * r;
          if (act && c < by) Z[kx * zs + (c ^ (kx & 7))] = cmul(v[0][r], axy.post[(size_t)ell * by + c]);
        }
      }
      __syncthreads();
      for (int c0 = 0; c0 < by; c0 += G) {
        const int c = c0 + g;
        const bool act = c < by;
        float2 v[1][E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int kx = t + T * r;
          v[0][r] = (act && kx < mx) ? cmul(Z[kx * zs + (c ^ (kx & 7))], axx.pre[(size_t)ell * mx + kx])
                                     : make_float2(0.f, 0.f);
        }
        block_fft<P, E, 1, -1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
        for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], axx.kspec[(size_t)ell * P + t + T * r]);
        block_fft<P, E, 1, +1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int a = t + T * r;
          if (act && a < bx) tile[a * ts + c * TL + (j ^ (a & 3))] = cmul(v[0][r], axx.post[(size_t)ell * bx + a]);
        }
      }
      __syncthreads();
    }
    float2* out = w + (size_t)blk * B * L + ell0;
    for (int idx = threadIdx.x; idx < B * TL; idx += blockDim.x) {
      const int b = idx / TL, jj = idx % TL, a = b / by, c = b % by;
      if (ell0 + jj < L) out[(size_t)b * L + jj] = tile[a * ts + c * TL + (jj ^ (a & 3))];
    }
    __syncthreads();
  }
}

template <int P>
static int czt_space_ura_P(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  constexpr int E = ura_e<P>::value;
  constexpr int T = P / E;
  constexpr int NTH = T >= 256 ? T : 256;
  constexpr int G = NTH / T;
  constexpr int TL = 4;
  const fbst_info& in = p->info;
  const fbst_axis_tables& axx = p->ax[0];
  const fbst_axis_tables& axy = p->same_axes ? p->ax[0] : p->ax[1];
  const size_t zs = ((size_t)axy.Ba + 7) / 8 * 8 + 8, ts = (size_t)axy.Ba * TL + 2;  // as in the kernel
  const size_t smem = sizeof(float2) * ((size_t)G * fft_smem_elems<float2>(P) + (size_t)axx.Ma * zs +
                                        (size_t)axx.Ba * ts);
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_czt_space_ura<P, TL, NTH>));
  const long long items = (long long)((in.L + TL - 1) / TL) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_czt_space_ura<P, TL, NTH>, NTH, smem));
  k_czt_space_ura<P, TL, NTH><<<grid, NTH, smem, s>>>(yhat, w, axx, axy, p->tw32, in.L, nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// ---------------------------------------------------------------------------------------------
// Non-uniform linear array (Sec. IX, Eq. (16)): the element sum of each frequency as a type-1
// NUFFT (tables from plan.cu). Work item = G consecutive frequencies of one block, one transform
// group of T = NF/E threads per frequency: zero the grid (real and imaginary parts in separate
// shared arrays, so the atomics of neighbouring points fall on different banks), spread every
// element's yhat[m, ell] onto its W grid points with shared-memory atomics, the W kernel weights
// evaluated in FP32 from the point's offset to its first grid point (the table keeps that offset to
// about 5e-7), take the unnormalised inverse-sign FFT of the grid in registers, and read beam b at
// mode b - B/2 times its deconvolution factor; the [B][G] tile leaves in G-frequency runs.
// ---------------------------------------------------------------------------------------------
template <int NF, int E, int G>
__global__ void __launch_bounds__(G * (NF / E))
k_nufft_space(const float2* __restrict__ yhat, float2* __restrict__ w, const int* __restrict__ j0,
              const float* __restrict__ dg, const float* __restrict__ deconv, const float2* __restrict__ tw, int M,
              int B, int L, int W, float beta, int nblk) {
  constexpr int T = NF / E;
  static_assert(T <= 32 || G <= 15, "named barriers 1..15, one per transform group");
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  float2* fbuf = sm + g * NF;                       // the FFT's exchange buffer ...
  float* gre = reinterpret_cast<float*>(fbuf);      // ... first holds the grid: real parts
  float* gim = gre + NF;                            //     and imaginary parts
  float2* tile = sm + G * NF;  // [B][G + 1]
  const float inv_half = 2.0f / W;
  long long it0, it1;
  my_range((long long)((L + G - 1) / G) * nblk, &it0, &it1);
  for (long long it = it0; it < it1; ++it) {
    const int lt = (int)(it / nblk), blk = (int)(it % nblk);
    const int ell0 = lt * G, ell = ell0 + g, ellc = ell < L ? ell : L - 1;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      gre[t + T * r] = 0.f;
      gim[t + T * r] = 0.f;
    }
    fft_sync<T>(1 + g);
    const float2* row = yhat + ((size_t)blk * L + ellc) * M;
    const int* jr = j0 + (size_t)ellc * M;
    const float* dr = dg + (size_t)ellc * M;
    for (int m = t; m < M; m += T) {
      const float2 c = row[m];
      const int jb = jr[m];
      const float d = dr[m];
      for (int q = 0; q < W; ++q) {
        const float z = ((float)q - d) * inv_half, z2 = z * z;
        // sqrt(1 - z^2) - 1 written as -z^2 / (1 + sqrt(1 - z^2)): no cancellation, so the
        // exponent keeps its relative precision and the weight about 1e-7 absolute.
        const float k = z2 < 1.f ? expf(-beta * z2 / (1.f + sqrtf(1.f - z2))) : 0.f;
        const int j = (jb + q) & (NF - 1);
        atomicAdd(&gre[j], c.x * k);
        atomicAdd(&gim[j], c.y * k);
      }
    }
    fft_sync<T>(1 + g);
    float2 v[1][E];
#pragma unroll
    for (int r = 0; r < E; ++r) v[0][r] = make_float2(gre[t + T * r], gim[t + T * r]);
    fft_sync<T>(1 + g);
    block_fft<NF, E, 1, +1>(v, fbuf, tw, t, 1 + g);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int k = t + T * r;
      const int b = (k < NF / 2 ? k : k - NF) + B / 2;
      if (b >= 0 && b < B) tile[b * (G + 1) + g] = cscale(v[0][r], deconv[b]);
    }
    __syncthreads();
    float2* out = w + (size_t)blk * B * L + ell0;
    for (int idx = threadIdx.x; idx < B * G; idx += blockDim.x) {
      const int b = idx / G, gg = idx % G;
      if (ell0 + gg < L) out[(size_t)b * L + gg] = tile[b * (G + 1) + gg];
    }
    __syncthreads();
  }
}

template <int NF>
static int run_nufft(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  constexpr int E = NF >= 512 ? 16 : 8;
  constexpr int T = NF / E;
  constexpr int G = T >= 256 ? 2 : (T >= 128 ? 4 : (T >= 32 ? 8 : (T >= 8 ? 8 : 16)));
  const fbst_info& in = p->info;
  const size_t smem = sizeof(float2) * ((size_t)G * NF + (size_t)in.B * (G + 1));
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_nufft_space<NF, E, G>));
  const long long items = (long long)((in.L + G - 1) / G) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_nufft_space<NF, E, G>, G * T, smem));
  k_nufft_space<NF, E, G><<<grid, G * T, smem, s>>>(yhat, w, p->nu_j0, p->nu_dg, p->nu_deconv, p->tw32, in.M, in.B,
                                                    in.L, p->nu_w, (float)nufft_beta(p->nu_w), nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

static int launch_space_nufft(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  switch (p->nu_nf) {
    case 16: return run_nufft<16>(p, yhat, w, nblk, s);
    case 32: return run_nufft<32>(p, yhat, w, nblk, s);
    case 64: return run_nufft<64>(p, yhat, w, nblk, s);
    case 128: return run_nufft<128>(p, yhat, w, nblk, s);
    case 256: return run_nufft<256>(p, yhat, w, nblk, s);
    case 512: return run_nufft<512>(p, yhat, w, nblk, s);
    case 1024: return run_nufft<1024>(p, yhat, w, nblk, s);
    case 2048: return run_nufft<2048>(p, yhat, w, nblk, s);
    case 4096: return run_nufft<4096>(p, yhat, w, nblk, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------------------------
// Non-uniform rectangular array (Sec. IX, Eq. (16) with both coordinates off the grid): the element
// sum of each frequency as a two-dimensional type-1 NUFFT. The oversampled grid has NFX x NFY
// points (NFX >= 2 bx, NFY >= 2 by); element m lands at grid coordinates (gx, gy) = (NFX 2 kappa
// x_m / bx, NFY 2 kappa y_m / by) (tables from plan.cu, one per axis) and is spread over W x W
// points with the product of the two one-dimensional kernels; the positions move independently in
// both axes, so the spreading does not separate into two one-dimensional passes. Then the 2-D
// unnormalised inverse-sign FFT: an NFY-point FFT along every row of the grid, and an NFX-point
// FFT along the by columns whose y-modes are beams; beam (bu, bv) (b = bu by + bv) is read at mode
// (bu - bx/2, bv - by/2) times the two axes' deconvolution factors. A CTA takes G consecutive
// frequencies of one block in turn; the [B][G] tile leaves in G-frequency runs. The grid rows are
// padded by one float (NFY + 1) so that the column FFT's strided loads fall on distinct banks.
// FFT groups: T = min(32, NF/2) threads (inside one warp: warp barriers), E = NF/T points each;
// every group makes the same number of transforms (a group past the last row or column transforms
// zeros and stores nothing), as the warp barriers need.
// ---------------------------------------------------------------------------------------------
constexpr int kNu2Threads = 256;
constexpr int kNu2G = 4;

template <int NF> struct nu2_shape {
  static constexpr int T = NF / 2 < 32 ? NF / 2 : 32;
  static constexpr int E = NF / T;
};

template <int NFX, int NFY>
__global__ void __launch_bounds__(kNu2Threads)
k_nufft_space_2d(const float2* __restrict__ yhat, float2* __restrict__ w, const int* __restrict__ j0x,
                 const float* __restrict__ dgx, const int* __restrict__ j0y, const float* __restrict__ dgy,
                 const float* __restrict__ deconv_x, const float* __restrict__ deconv_y,
                 const float2* __restrict__ tw, int M, int bx, int by, int L, int W, float beta, int nblk) {
  constexpr int RS = NFY + 1;  // padded row stride of the grid
  constexpr int TY = nu2_shape<NFY>::T, EY = nu2_shape<NFY>::E;
  constexpr int TX = nu2_shape<NFX>::T, EX = nu2_shape<NFX>::E;
  constexpr int GY = kNu2Threads / TY, GX = kNu2Threads / TX;  // FFT groups per CTA
  constexpr int XB = (GY * NFY > GX * NFX) ? GY * NFY : GX * NFX;
  extern __shared__ float2 sm[];
  float* gre = reinterpret_cast<float*>(sm);
  float* gim = gre + NFX * RS;
  float2* xbuf = sm + NFX * RS;   // FFT exchange buffers (after the two float planes)
  float2* tile = xbuf + XB;       // [B][kNu2G + 1]
  const int B = bx * by;
  const int tid = threadIdx.x;
  const float inv_half = 2.0f / W;
  long long it0, it1;
  my_range((long long)((L + kNu2G - 1) / kNu2G) * nblk, &it0, &it1);
  for (long long it = it0; it < it1; ++it) {
    const int lt = (int)(it / nblk), blk = (int)(it % nblk);
    const int ell0 = lt * kNu2G;
    for (int g = 0; g < kNu2G && ell0 + g < L; ++g) {
      const int ell = ell0 + g;
      for (int i = tid; i < NFX * RS; i += kNu2Threads) {
        gre[i] = 0.f;
        gim[i] = 0.f;
      }
      __syncthreads();
      const float2* row = yhat + ((size_t)blk * L + ell) * M;
      const int* jxr = j0x + (size_t)ell * M;
      const int* jyr = j0y + (size_t)ell * M;
      const float* dxr = dgx + (size_t)ell * M;
      const float* dyr = dgy + (size_t)ell * M;
      for (int m = tid; m < M; m += kNu2Threads) {
        const float2 c = row[m];
        const int jx = jxr[m], jy = jyr[m];
        const float dx = dxr[m], dy = dyr[m];
        float ky[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float z = ((float)q - dy) * inv_half, z2 = z * z;
          ky[q] = (q < W && z2 < 1.f) ? expf(-beta * z2 / (1.f + sqrtf(1.f - z2))) : 0.f;
        }
        for (int qx = 0; qx < W; ++qx) {
          const float z = ((float)qx - dx) * inv_half, z2 = z * z;
          const float kx = z2 < 1.f ? expf(-beta * z2 / (1.f + sqrtf(1.f - z2))) : 0.f;
          const float cr = c.x * kx, ci = c.y * kx;
          const int base = ((jx + qx) & (NFX - 1)) * RS;
#pragma unroll
          for (int qy = 0; qy < 16; ++qy) {
            if (qy < W) {
              const int j = base + ((jy + qy) & (NFY - 1));
              atomicAdd(&gre[j], cr * ky[qy]);
              atomicAdd(&gim[j], ci * ky[qy]);
            }
          }
        }
      }
      __syncthreads();
      {  // NFY-point transforms along the NFX rows
        const int grp = tid / TY, t = tid % TY;
        float2* fb = xbuf + grp * NFY;
        for (int r0 = 0; r0 < NFX; r0 += GY) {
          const int rr = r0 + grp;
          float2 v[1][EY];
#pragma unroll
          for (int r = 0; r < EY; ++r) {
            const int j = t + TY * r;
            v[0][r] = rr < NFX ? make_float2(gre[rr * RS + j], gim[rr * RS + j]) : make_float2(0.f, 0.f);
          }
          block_fft<NFY, EY, 1, +1>(v, fb, tw, t, 1 + (grp & 15));
          if (rr < NFX) {
#pragma unroll
            for (int r = 0; r < EY; ++r) {
              const int j = t + TY * r;
              gre[rr * RS + j] = v[0][r].x;
              gim[rr * RS + j] = v[0][r].y;
            }
          }
        }
      }
      __syncthreads();
      {  // NFX-point transforms along the by columns that hold beams
        const int grp = tid / TX, t = tid % TX;
        float2* fb = xbuf + grp * NFX;
        for (int c0 = 0; c0 < by; c0 += GX) {
          const int bv = c0 + grp;
          const int col = ((bv - by / 2) + NFY) & (NFY - 1);
          float2 v[1][EX];
#pragma unroll
          for (int r = 0; r < EX; ++r) {
            const int j = t + TX * r;
            v[0][r] = bv < by ? make_float2(gre[j * RS + col], gim[j * RS + col]) : make_float2(0.f, 0.f);
          }
          block_fft<NFX, EX, 1, +1>(v, fb, tw, t, 1 + (grp & 15));
          if (bv < by) {
            const float sy = deconv_y[bv];
#pragma unroll
            for (int r = 0; r < EX; ++r) {
              const int k = t + TX * r;
              const int bu = (k < NFX / 2 ? k : k - NFX) + bx / 2;
              if (bu >= 0 && bu < bx) tile[(bu * by + bv) * (kNu2G + 1) + g] = cscale(v[0][r], deconv_x[bu] * sy);
            }
          }
        }
      }
      __syncthreads();
    }
    float2* out = w + (size_t)blk * B * L + ell0;
    for (int idx = tid; idx < B * kNu2G; idx += kNu2Threads) {
      const int b = idx / kNu2G, gg = idx % kNu2G;
      if (ell0 + gg < L) out[(size_t)b * L + gg] = tile[b * (kNu2G + 1) + gg];
    }
    __syncthreads();
  }
}

template <int NFX, int NFY>
static int run_nufft_2d(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  constexpr int RS = NFY + 1;
  constexpr int GY = kNu2Threads / nu2_shape<NFY>::T, GX = kNu2Threads / nu2_shape<NFX>::T;
  constexpr int XB = (GY * NFY > GX * NFX) ? GY * NFY : GX * NFX;
  const fbst_info& in = p->info;
  if (p->nu_w > 16) return FBST_ERR_UNSUPPORTED;
  const size_t smem = sizeof(float) * 2 * NFX * RS + sizeof(float2) * ((size_t)XB + (size_t)in.B * (kNu2G + 1));
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_nufft_space_2d<NFX, NFY>));
  const long long items = (long long)((in.L + kNu2G - 1) / kNu2G) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_nufft_space_2d<NFX, NFY>, kNu2Threads, smem));
  k_nufft_space_2d<NFX, NFY><<<grid, kNu2Threads, smem, s>>>(
      yhat, w, p->nu_j0, p->nu_dg, p->nu_j0y, p->nu_dgy, p->nu_deconv, p->nu_deconv_y, p->tw32, in.M, p->geom.bx,
      p->geom.by, in.L, p->nu_w, (float)nufft_beta(p->nu_w), nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

template <int NFX>
static int launch_nufft_2d_x(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  switch (p->nu_nfy) {
    case 16: return run_nufft_2d<NFX, 16>(p, yhat, w, nblk, s);
    case 32: return run_nufft_2d<NFX, 32>(p, yhat, w, nblk, s);
    case 64: return run_nufft_2d<NFX, 64>(p, yhat, w, nblk, s);
    case 128: return run_nufft_2d<NFX, 128>(p, yhat, w, nblk, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

static int launch_space_nufft_2d(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  switch (p->nu_nf) {
    case 16: return launch_nufft_2d_x<16>(p, yhat, w, nblk, s);
    case 32: return launch_nufft_2d_x<32>(p, yhat, w, nblk, s);
    case 64: return launch_nufft_2d_x<64>(p, yhat, w, nblk, s);
    case 128: return launch_nufft_2d_x<128>(p, yhat, w, nblk, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

static int czt_space(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, unsigned* wmax, cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  if (p->nu_nf && p->nu_nfy) return launch_space_nufft_2d(p, yhat, w, nblk, s);
  if (p->nu_nf) return launch_space_nufft(p, yhat, w, nblk, s);
  if (p->geom.kind == FBST_ULA) {
    job_list<space_job> jl;
    jl.n = 1;
    jl.job[0] = make_space_job(p, yhat, w, nblk);
    if (wmax) {
      FBST_CUDA_TRY(cudaMemsetAsync(wmax, 0, sizeof(unsigned) * nblk, s));
      jl.job[0].wmax = wmax;
    }
    const fft_shape sh = space_shape(p);
    jl.total = space_items(jl.job[0], sh, p->info.P_space_x);
    return launch_space_jobs(jl, p->info.P_space_x, sh, p->ax[0].Ba, p->tw32, s);
  }
  if (p->info.P_space_x != p->info.P_space_y) return FBST_ERR_UNSUPPORTED;
  switch (p->info.P_space_x) {
    case 16: return czt_space_ura_P<16>(p, yhat, w, nblk, s);
    case 32: return czt_space_ura_P<32>(p, yhat, w, nblk, s);
    case 64: return czt_space_ura_P<64>(p, yhat, w, nblk, s);
    case 128: return czt_space_ura_P<128>(p, yhat, w, nblk, s);
    case 256: return czt_space_ura_P<256>(p, yhat, w, nblk, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

int launch_czt_space(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  return czt_space(p, yhat, w, nblk, nullptr, s);
}

int launch_czt_space_scaled(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, int blk0,
                            cudaStream_t s) {
  if (p->tc_wmax_stage1 && (blk0 < 0 || blk0 + nblk > p->band.max_blocks)) return FBST_ERR_INVALID;
  return czt_space(p, yhat, w, nblk, p->tc_wmax_stage1 ? p->tc_wmax + blk0 : nullptr, s);
}

}  // namespace fbst
