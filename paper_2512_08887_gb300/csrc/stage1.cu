// Stage 1 of the FBST, the "fan" chirp-z of Sec. IV (App. B for rectangular arrays):
//   yhat[m, ell] = sum_n y[m, n] exp(-2*pi*i*eps*ell'*n/L)                     (temporal chirp-z)
//   w[b, ell]    = sum_m yhat[m, ell] exp(2*pi*i*kappa_ell*(u_b.p_m)),         (spatial chirp-z)
//   kappa_ell = rho*(1/fb + eps*ell'/L),
// both evaluated by Bluestein: chirp premultiply, FFT, multiply by the precomputed spectrum of
// the chirp kernel, inverse FFT, chirp postmultiply (tables built in plan.cu).
//
// Layout: y [blk][M][N] -> yhat [blk][L][M] -> w [blk][B][L]. Each transpose happens in shared
// memory: a work item is a few consecutive elements (temporal) or frequencies (spatial) of one
// block, written back as 32-byte runs so every global store fills whole sectors.
//
// Work distribution: the grid holds exactly the CTAs that fit on the GPU at once (occupancy x SM
// count) and CTA c processes the contiguous range [c*I/G, (c+1)*I/G) of the I flattened work
// items, so no partial last wave idles the machine; per-frequency tables are reloaded only when
// the range crosses to the next frequency tile.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"

namespace fbst {

// Elements per thread for a Stockham transform of size P in the FP32 hot kernels.
template <int P> struct hot_e { static constexpr int value = P >= 2048 ? 16 : (P >= 8 ? 8 : 2); };

__device__ __forceinline__ void my_range(long long items, long long* begin, long long* end) {
  const long long G = gridDim.x, c = blockIdx.x;
  *begin = items * c / G;
  *end = items * (c + 1) / G;
}

// Resident CTAs of `kernel` on the current device for the given block size and shared memory.
template <typename K>
static int resident_ctas(K kernel, int threads, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return sms * per_sm;
}

static int grid_for_items(long long items, int slots) {
  return (int)std::max<long long>(1, std::min<long long>(items, slots));
}

// ---------------------------------------------------------------------------------------------
// Temporal chirp-z. Work item = (block, tile of TS consecutive elements); one Stockham group per
// element. Output k = h*Lh + i comes from inverse transform h (S of them share one forward one).
// ---------------------------------------------------------------------------------------------
template <int P, int TS>
__global__ void __launch_bounds__(TS * (P / hot_e<P>::value))
k_czt_time(const float2* __restrict__ y, float2* __restrict__ yhat, const float2* __restrict__ pre,
           const float2* __restrict__ gspec, const float2* __restrict__ post, const float2* __restrict__ tw,
           int M, int N, int L, int S, int nblk) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int SB = fft_smem_elems<float2>(P);
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  const int Lh = L / S;
  const int ntile = (M + TS - 1) / TS;
  float2* fbuf = sm + g * SB;
  float2* tile = sm + TS * SB;  // [Lh][TS]
  long long it0, it1;
  my_range((long long)ntile * nblk, &it0, &it1);
  for (long long it = it0; it < it1; ++it) {
    const int blk = (int)(it / ntile), m0 = (int)(it % ntile) * TS;
    const int m = m0 + g;
    const float2* yrow = y + ((size_t)blk * M + (m < M ? m : M - 1)) * N;
    float2 v[1][E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int n = t + T * r;
      v[0][r] = (n < N && m < M) ? cmul(yrow[n], pre[n]) : make_float2(0.f, 0.f);
    }
    block_fft<P, E, 1, -1>(v, fbuf, tw, t);
    for (int h = 0; h < S; ++h) {
      float2 u[1][E];
#pragma unroll
      for (int r = 0; r < E; ++r) u[0][r] = cmul(v[0][r], gspec[h * P + t + T * r]);
      block_fft<P, E, 1, +1>(u, fbuf, tw, t);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = t + T * r;
        if (i < Lh) tile[i * TS + g] = cmul(u[0][r], post[h * Lh + i]);
      }
      __syncthreads();
      float2* out = yhat + ((size_t)blk * L + (size_t)h * Lh) * M + m0;
      for (int idx = threadIdx.x; idx < Lh * TS; idx += blockDim.x) {
        const int i = idx / TS, gg = idx % TS;
        if (m0 + gg < M) out[(size_t)i * M + gg] = tile[idx];
      }
      __syncthreads();
    }
  }
}

template <int P>
static int czt_time_P(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk, cudaStream_t s) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int TS = T >= 256 ? 2 : (T >= 64 ? 4 : (T >= 16 ? 8 : 16));
  const fbst_info& in = p->info;
  const int Lh = in.L / in.S_time;
  const size_t smem = sizeof(float2) * ((size_t)TS * fft_smem_elems<float2>(P) + (size_t)Lh * TS);
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_czt_time<P, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long items = (long long)((in.M + TS - 1) / TS) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_czt_time<P, TS>, TS * T, smem));
  k_czt_time<P, TS><<<grid, TS * T, smem, s>>>(y, yhat, p->pre_t, p->gspec_t, p->post_t, p->tw32, in.M, in.N,
                                               in.L, in.S_time, nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int launch_czt_time(const fbst_plan_s* p, const float2* y, float2* yhat, int nblk, cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  switch (p->info.P_time) {
    case 16: return czt_time_P<16>(p, y, yhat, nblk, s);
    case 32: return czt_time_P<32>(p, y, yhat, nblk, s);
    case 64: return czt_time_P<64>(p, y, yhat, nblk, s);
    case 128: return czt_time_P<128>(p, y, yhat, nblk, s);
    case 256: return czt_time_P<256>(p, y, yhat, nblk, s);
    case 512: return czt_time_P<512>(p, y, yhat, nblk, s);
    case 1024: return czt_time_P<1024>(p, y, yhat, nblk, s);
    case 2048: return czt_time_P<2048>(p, y, yhat, nblk, s);
    case 4096: return czt_time_P<4096>(p, y, yhat, nblk, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

// ---------------------------------------------------------------------------------------------
// Spatial chirp-z of a linear array. Work item = (tile of TL consecutive frequencies, block),
// ordered tile-major so a CTA's range mostly shares one tile: the per-frequency chirps and kernel
// spectrum stay in registers until the tile changes.
// ---------------------------------------------------------------------------------------------
template <int P, int TL>
__global__ void __launch_bounds__(TL * (P / hot_e<P>::value))
k_czt_space_ula(const float2* __restrict__ yhat, float2* __restrict__ w, const float2* __restrict__ pre,
                const float2* __restrict__ kspec, const float2* __restrict__ post, const float2* __restrict__ tw,
                int M, int B, int L, int nblk) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int SB = fft_smem_elems<float2>(P);
  extern __shared__ float2 sm[];
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  float2* fbuf = sm + g * SB;
  float2* tile = sm + TL * SB;  // [B][TL]
  const int ntile = (L + TL - 1) / TL;
  long long it0, it1;
  my_range((long long)ntile * nblk, &it0, &it1);
  int cur = -1;
  float2 pr[E], ks[E], po[E];
  for (long long it = it0; it < it1; ++it) {
    const int lt = (int)(it / nblk), blk = (int)(it % nblk);
    const int ell0 = lt * TL;
    const int ell = ell0 + g;
    const int ellc = ell < L ? ell : L - 1;
    if (lt != cur) {
      cur = lt;
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = t + T * r;
        pr[r] = i < M ? pre[(size_t)ellc * M + i] : make_float2(0.f, 0.f);
        ks[r] = kspec[(size_t)ellc * P + i];
        po[r] = i < B ? post[(size_t)ellc * B + i] : make_float2(0.f, 0.f);
      }
    }
    const float2* row = yhat + ((size_t)blk * L + ellc) * M;
    float2 v[1][E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = t + T * r;
      v[0][r] = i < M ? cmul(row[i], pr[r]) : make_float2(0.f, 0.f);
    }
    block_fft<P, E, 1, -1>(v, fbuf, tw, t);
#pragma unroll
    for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], ks[r]);
    block_fft<P, E, 1, +1>(v, fbuf, tw, t);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int b = t + T * r;
      if (b < B) tile[b * TL + g] = cmul(v[0][r], po[r]);
    }
    __syncthreads();
    float2* out = w + (size_t)blk * B * L + ell0;
    for (int idx = threadIdx.x; idx < B * TL; idx += blockDim.x) {
      const int b = idx / TL, gg = idx % TL;
      if (ell0 + gg < L) out[(size_t)b * L + gg] = tile[idx];
    }
    __syncthreads();
  }
}

template <int P>
static int czt_space_ula_P(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int TL = T >= 256 ? 2 : (T >= 64 ? 4 : (T >= 16 ? 8 : 16));
  const fbst_info& in = p->info;
  const fbst_axis_tables& ax = p->ax[0];
  const size_t smem = sizeof(float2) * ((size_t)TL * fft_smem_elems<float2>(P) + (size_t)ax.Ba * TL);
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_czt_space_ula<P, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long items = (long long)((in.L + TL - 1) / TL) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_czt_space_ula<P, TL>, TL * T, smem));
  k_czt_space_ula<P, TL><<<grid, TL * T, smem, s>>>(yhat, w, ax.pre, ax.kspec, ax.post, p->tw32, ax.Ma, ax.Ba,
                                                    in.L, nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// ---------------------------------------------------------------------------------------------
// Spatial chirp-z of an mx-by-my rectangular array (App. B): for each frequency, a chirp-z along
// y (my -> by) for every row kx, then along x (mx -> bx) for every beam column c, both in shared
// memory. Work item = (tile of TL consecutive frequencies, block). Both axes use size-P transforms.
// ---------------------------------------------------------------------------------------------
template <int P, int TL, int NTH>
__global__ void __launch_bounds__(NTH)
k_czt_space_ura(const float2* __restrict__ yhat, float2* __restrict__ w, fbst_axis_tables axx,
                fbst_axis_tables axy, const float2* __restrict__ tw, int L, int nblk) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int G = NTH / T;  // concurrent transforms
  constexpr int SB = fft_smem_elems<float2>(P);
  extern __shared__ float2 sm[];
  const int mx = axx.Ma, bx = axx.Ba, my = axy.Ma, by = axy.Ba;
  const int M = mx * my, B = bx * by;
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  float2* fbuf = sm + g * SB;
  float2* Z = sm + G * SB;      // [mx][by]
  float2* tile = Z + mx * by;   // [B][TL]
  const int ntile = (L + TL - 1) / TL;
  long long it0, it1;
  my_range((long long)ntile * nblk, &it0, &it1);
  for (long long it = it0; it < it1; ++it) {
    const int lt = (int)(it / nblk), blk = (int)(it % nblk);
    const int ell0 = lt * TL;
    for (int j = 0; j < TL; ++j) {
      const int ell = min(ell0 + j, L - 1);
      const float2* src = yhat + ((size_t)blk * L + ell) * M;
      // Along y: rows kx.
      for (int kx0 = 0; kx0 < mx; kx0 += G) {
        const int kx = kx0 + g;
        const bool act = kx < mx;
        float2 v[1][E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int ky = t + T * r;
          v[0][r] = (act && ky < my) ? cmul(src[kx * my + ky], axy.pre[(size_t)ell * my + ky]) : make_float2(0.f, 0.f);
        }
        block_fft<P, E, 1, -1>(v, fbuf, tw, t);
#pragma unroll
        for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], axy.kspec[(size_t)ell * P + t + T * r]);
        block_fft<P, E, 1, +1>(v, fbuf, tw, t);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int c = t + T * r;
          if (act && c < by) Z[kx * by + c] = cmul(v[0][r], axy.post[(size_t)ell * by + c]);
        }
      }
      __syncthreads();
      // Along x: beam columns c.
      for (int c0 = 0; c0 < by; c0 += G) {
        const int c = c0 + g;
        const bool act = c < by;
        float2 v[1][E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int kx = t + T * r;
          v[0][r] = (act && kx < mx) ? cmul(Z[kx * by + c], axx.pre[(size_t)ell * mx + kx]) : make_float2(0.f, 0.f);
        }
        block_fft<P, E, 1, -1>(v, fbuf, tw, t);
#pragma unroll
        for (int r = 0; r < E; ++r) v[0][r] = cmul(v[0][r], axx.kspec[(size_t)ell * P + t + T * r]);
        block_fft<P, E, 1, +1>(v, fbuf, tw, t);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const int a = t + T * r;
          if (act && a < bx) tile[(a * by + c) * TL + j] = cmul(v[0][r], axx.post[(size_t)ell * bx + a]);
        }
      }
      __syncthreads();
    }
    float2* out = w + (size_t)blk * B * L + ell0;
    for (int idx = threadIdx.x; idx < B * TL; idx += blockDim.x) {
      const int b = idx / TL, jj = idx % TL;
      if (ell0 + jj < L) out[(size_t)b * L + jj] = tile[idx];
    }
    __syncthreads();
  }
}

template <int P>
static int czt_space_ura_P(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  constexpr int E = hot_e<P>::value;
  constexpr int T = P / E;
  constexpr int NTH = T >= 256 ? T : 256;
  constexpr int G = NTH / T;
  constexpr int TL = 4;
  const fbst_info& in = p->info;
  const fbst_axis_tables& axx = p->ax[0];
  const fbst_axis_tables& axy = p->same_axes ? p->ax[0] : p->ax[1];
  const size_t smem = sizeof(float2) * ((size_t)G * fft_smem_elems<float2>(P) + (size_t)axx.Ma * axy.Ba +
                                        (size_t)in.B * TL);
  if (smem > 227 * 1024) return FBST_ERR_UNSUPPORTED;
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_czt_space_ura<P, TL, NTH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long items = (long long)((in.L + TL - 1) / TL) * nblk;
  const int grid = grid_for_items(items, resident_ctas(k_czt_space_ura<P, TL, NTH>, NTH, smem));
  k_czt_space_ura<P, TL, NTH><<<grid, NTH, smem, s>>>(yhat, w, axx, axy, p->tw32, in.L, nblk);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int launch_czt_space(const fbst_plan_s* p, const float2* yhat, float2* w, int nblk, cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  if (p->geom.kind == FBST_ULA) {
    switch (p->info.P_space_x) {
      case 16: return czt_space_ula_P<16>(p, yhat, w, nblk, s);
      case 32: return czt_space_ula_P<32>(p, yhat, w, nblk, s);
      case 64: return czt_space_ula_P<64>(p, yhat, w, nblk, s);
      case 128: return czt_space_ula_P<128>(p, yhat, w, nblk, s);
      case 256: return czt_space_ula_P<256>(p, yhat, w, nblk, s);
      case 512: return czt_space_ula_P<512>(p, yhat, w, nblk, s);
      case 1024: return czt_space_ula_P<1024>(p, yhat, w, nblk, s);
      case 2048: return czt_space_ula_P<2048>(p, yhat, w, nblk, s);
      case 4096: return czt_space_ula_P<4096>(p, yhat, w, nblk, s);
      default: return FBST_ERR_UNSUPPORTED;
    }
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

}  // namespace fbst
