// Stage 2 of the FBST (Sec. V): beta_b = A_b^{-1} w_b, bhat_b = F_u beta_b.
//
// k_stage2_gs fuses, per (beam, block) work item: the Gohberg-Semencul product (gs.cuh, six
// transforms of size P_gs >= 2L-1), optionally one FP32 refinement step (beta += GS(w - A_b beta),
// the Toeplitz product through its circulant embedding), and the reconstruction chirp-z of F_u
// (Eq. (7)) by Bluestein with S_rec input splits (S_rec forward transforms of size P_rec summed in
// frequency, one inverse). beta never leaves shared memory; the only HBM traffic is w in and bhat
// out. Work items of all jobs of a launch are flattened beam-major and split evenly over the
// resident CTAs; a CTA keeps the current beam's spectra in registers.
//
// k_dense_fp32 applies the precomputed G_b = F_u A_b^{-1} (N x L, Sec. III-B) as a batched
// complex GEMM over blocks on the FP32 CUDA cores.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "gs.cuh"
#include "launch_util.cuh"

namespace fbst {

template <int P> struct gs_e { static constexpr int value = P >= 4096 ? 16 : (P >= 16 ? 8 : 2); };

template <int PG, int PR, int SR, bool IR>
__global__ void __launch_bounds__(PG / gs_e<PG>::value)
k_stage2_gs(const __grid_constant__ job_list<gs_job> jl, const float2* __restrict__ tw) {
  constexpr int EG = gs_e<PG>::value;
  constexpr int T = PG / EG;
  constexpr int ER = PR / T;
  static_assert(ER >= 2 && ER * T == PR, "reconstruction transform must span the same threads");
  constexpr int SBG = fft_smem_elems<float2>(PG);
  extern __shared__ float2 sm[];
  float2* beta_s = sm + 2 * SBG;  // [L]
  const int t = threadIdx.x;
  long long it0, it1;
  my_range(jl.total, &it0, &it1);
  int j = 0, cur_j = -1, b_cur = -1;
  float2 X[EG], Vv[EG];

  for (long long it = it0; it < it1; ++it) {
    while (j + 1 < jl.n && jl.job[j + 1].first <= it) ++j;
    const gs_job& J = jl.job[j];
    const int B = J.B, L = J.L, N = J.N, nblk = J.nblk;
    const int Lr = L / SR;
    const long long li = it - J.first;
    const int b = (int)(li / nblk), blk = (int)(li % nblk);
    if (b != b_cur || j != cur_j) {
      b_cur = b;
      cur_j = j;
      const float2* xv = J.XV + (size_t)b * 2 * PG;
#pragma unroll
      for (int r = 0; r < EG; ++r) {
        X[r] = xv[t + T * r];
        Vv[r] = xv[PG + t + T * r];
      }
    }
    const float2* wb = J.w + ((size_t)blk * B + b) * L;
    float2 v[EG];
#pragma unroll
    for (int r = 0; r < EG; ++r) {
      const int i = t + T * r;
      v[r] = i < L ? wb[i] : make_float2(0.f, 0.f);
    }
    gs_apply<PG, EG>(v, X, Vv, sm, tw, t, L);
    if constexpr (IR) {
      // One refinement step: r = w - A beta (Toeplitz product through its circulant embedding),
      // beta += GS(r). The residual's rounding error lies mostly where A_b is small, which F_u
      // (whose rows are rows of F_b) does not see; the GS cancellation error is removed.
      const float2* As = J.Aspec + (size_t)b * PG;
      float2 a[1][EG];
#pragma unroll
      for (int r = 0; r < EG; ++r) a[0][r] = (t + T * r < L) ? v[r] : make_float2(0.f, 0.f);
      block_fft<PG, EG, 1, -1>(a, sm, tw, t);
#pragma unroll
      for (int r = 0; r < EG; ++r) a[0][r] = cmul(a[0][r], As[t + T * r]);
      block_fft<PG, EG, 1, +1>(a, sm, tw, t);
      float2 res[EG];
#pragma unroll
      for (int r = 0; r < EG; ++r) {
        const int i = t + T * r;
        res[r] = i < L ? csub(wb[i], a[0][r]) : make_float2(0.f, 0.f);
      }
      gs_apply<PG, EG>(res, X, Vv, sm, tw, t, L);
#pragma unroll
      for (int r = 0; r < EG; ++r) v[r] = cadd(v[r], res[r]);
    }
#pragma unroll
    for (int r = 0; r < EG; ++r) {
      const int i = t + T * r;
      if (i < L) beta_s[i] = v[r];
    }
    __syncthreads();
    // Reconstruction: bhat[n] = post[n] * IFFT( sum_h FFT(beta_h * pre_h) * Q_h )[n].
    float2 x[SR][ER];
#pragma unroll
    for (int h = 0; h < SR; ++h) {
#pragma unroll
      for (int r = 0; r < ER; ++r) {
        const int i = t + T * r;
        x[h][r] = i < Lr ? cmul(beta_s[h * Lr + i], J.pre_r[h * Lr + i]) : make_float2(0.f, 0.f);
      }
    }
    block_fft<PR, ER, SR, -1>(x, sm, tw, t);
    float2 R[1][ER];
#pragma unroll
    for (int r = 0; r < ER; ++r) {
      float2 acc = cmul(x[0][r], J.qspec[t + T * r]);
#pragma unroll
      for (int h = 1; h < SR; ++h) acc = cadd(acc, cmul(x[h][r], J.qspec[h * PR + t + T * r]));
      R[0][r] = acc;
    }
    block_fft<PR, ER, 1, +1>(R, sm, tw, t);
    float2* ob = J.bhat + ((size_t)blk * B + b) * N;
#pragma unroll
    for (int r = 0; r < ER; ++r) {
      const int n = t + T * r;
      if (n < N) ob[n] = cmul(R[0][r], J.post_r[n]);
    }
  }
}

template <int PG, int PR, int SR, bool IR>
static int run_gs(const job_list<gs_job>& jl, int max_L, const float2* tw, cudaStream_t s) {
  constexpr int T = PG / gs_e<PG>::value;
  const size_t smem = sizeof(float2) * (2 * (size_t)fft_smem_elems<float2>(PG) + max_L);
  if (smem > kMaxSmem) return FBST_ERR_UNSUPPORTED;
  FBST_TRY(allow_max_smem(k_stage2_gs<PG, PR, SR, IR>));
  const int grid = grid_for_items(jl.total, resident_ctas(k_stage2_gs<PG, PR, SR, IR>, T, smem));
  k_stage2_gs<PG, PR, SR, IR><<<grid, T, smem, s>>>(jl, tw);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

template <int PG, bool IR>
static int gs_PGI(const job_list<gs_job>& jl, int PR, int SR, int max_L, const float2* tw, cudaStream_t s) {
  if constexpr (gs_e<PG>::value >= 4) {
    if (2 * PR == PG && SR == 2) return run_gs<PG, PG / 2, 2, IR>(jl, max_L, tw, s);
    if (2 * PR == PG && SR == 1) return run_gs<PG, PG / 2, 1, IR>(jl, max_L, tw, s);
  }
  if (PR == PG && SR == 1) return run_gs<PG, PG, 1, IR>(jl, max_L, tw, s);
  if (PR == PG && SR == 2) return run_gs<PG, PG, 2, IR>(jl, max_L, tw, s);
  return FBST_ERR_UNSUPPORTED;
}

template <int PG>
static int gs_PG(const job_list<gs_job>& jl, int PR, int SR, bool IR, int max_L, const float2* tw, cudaStream_t s) {
  return IR ? gs_PGI<PG, true>(jl, PR, SR, max_L, tw, s) : gs_PGI<PG, false>(jl, PR, SR, max_L, tw, s);
}

int launch_gs_jobs(const job_list<gs_job>& jl, int PG, int PR, int SR, bool IR, int max_L, const float2* tw,
                   cudaStream_t s) {
  if (jl.total <= 0) return FBST_OK;
  switch (PG) {
    case 16: return gs_PG<16>(jl, PR, SR, IR, max_L, tw, s);
    case 32: return gs_PG<32>(jl, PR, SR, IR, max_L, tw, s);
    case 64: return gs_PG<64>(jl, PR, SR, IR, max_L, tw, s);
    case 128: return gs_PG<128>(jl, PR, SR, IR, max_L, tw, s);
    case 256: return gs_PG<256>(jl, PR, SR, IR, max_L, tw, s);
    case 512: return gs_PG<512>(jl, PR, SR, IR, max_L, tw, s);
    case 1024: return gs_PG<1024>(jl, PR, SR, IR, max_L, tw, s);
    case 2048: return gs_PG<2048>(jl, PR, SR, IR, max_L, tw, s);
    case 4096: return gs_PG<4096>(jl, PR, SR, IR, max_L, tw, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

gs_job make_gs_job(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk) {
  const fbst_info& in = p->info;
  return gs_job{w, bhat, p->XV, p->Aspec, p->pre_r, p->qspec_r, p->post_r, in.B, in.L, in.N, nblk, 0};
}

int launch_stage2_gs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  const fbst_info& in = p->info;
  job_list<gs_job> jl;
  jl.n = 1;
  jl.job[0] = make_gs_job(p, w, bhat, nblk);
  jl.total = (long long)in.B * nblk;
  return launch_gs_jobs(jl, in.P_gs, in.P_rec, in.S_rec, in.stage2 == FBST_STAGE2_GS_IR1, in.L, p->tw32, s);
}

// ---------------------------------------------------------------------------------------------
// Dense FP32 apply: bhat[blk][b][n] = sum_ell G[b][n][ell] * w[blk][b][ell] (w_stride = B), or with
// one right-hand side per block shared by every beam, w[blk][ell] (w_stride = 0: the nulling
// contraction). CTA tile: 64 samples x 64 blocks of one beam, K chunks of 32 through shared memory;
// each thread owns 4 x 4 outputs (samples tn + 16 i, blocks tb + 16 j), so a K step costs 8 shared
// loads for 16 complex multiply-adds. Each K chunk is summed in FP32 on its own and then added to the
// running sum (blocked accumulation: the rounding error grows with the chunk length plus the number
// of chunks, not with L).
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_dense_fp32(const float2* __restrict__ G, const float2* __restrict__ w, float2* __restrict__ bhat,
             int B, int N, int L, int nblk, int w_stride) {
  __shared__ float2 Gs[64][33];
  __shared__ float2 Ws[64][33];
  const int b = blockIdx.y, n0 = blockIdx.x * 64, blk0 = blockIdx.z * 64;
  const int tid = threadIdx.x, tn = tid & 15, tb = tid >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const float2* Gb = G + (size_t)b * N * L;
  const size_t wrow = w_stride ? (size_t)B * L : (size_t)L;   // elements between two blocks' rows
  const float2* wb = w + (w_stride ? (size_t)b * L : 0);
  for (int k0 = 0; k0 < L; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = tid + 256 * q, row = idx >> 5, col = idx & 31;
      const int n = n0 + row, k = k0 + col, blk = blk0 + row;
      Gs[row][col] = (n < N && k < L) ? Gb[(size_t)n * L + k] : make_float2(0.f, 0.f);
      Ws[row][col] = (blk < nblk && k < L) ? wb[(size_t)blk * wrow + k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float2 gv[4], wv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) gv[i] = Gs[tn + 16 * i][kk];
#pragma unroll
      for (int j = 0; j < 4; ++j) wv[j] = Ws[tb + 16 * j][kk];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          part[i][j].x = fmaf(gv[i].x, wv[j].x, fmaf(-gv[i].y, wv[j].y, part[i][j].x));
          part[i][j].y = fmaf(gv[i].x, wv[j].y, fmaf(gv[i].y, wv[j].x, part[i][j].y));
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].x += part[i][j].x;
        acc[i][j].y += part[i][j].y;
      }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int blk = blk0 + tb + 16 * j;
    if (blk >= nblk) continue;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int n = n0 + tn + 16 * i;
      if (n < N) bhat[((size_t)blk * B + b) * N + n] = acc[i][j];
    }
  }
}

int launch_dense_fp32_rhs(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, bool shared_rhs,
                          cudaStream_t s) {
  if (nblk <= 0) return FBST_OK;
  const fbst_info& in = p->info;
  const dim3 grid((in.N + 63) / 64, in.B, (nblk + 63) / 64);
  if (grid.z > 65535 || grid.y > 65535) return FBST_ERR_UNSUPPORTED;
  k_dense_fp32<<<grid, 256, 0, s>>>(p->G, w, bhat, in.B, in.N, in.L, nblk, shared_rhs ? 0 : 1);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int launch_stage2_dense_fp32(const fbst_plan_s* p, const float2* w, float2* bhat, int nblk, cudaStream_t s) {
  return launch_dense_fp32_rhs(p, w, bhat, nblk, false, s);
}

int stage2_launches(const fbst_plan_s* p, bool w_from_stage1) {
  switch (p->info.stage2) {
    case FBST_STAGE2_GS:
    case FBST_STAGE2_GS_IR1: return 1;
    case FBST_STAGE2_DENSE_FP32: return 1;
    case FBST_STAGE2_DENSE_TF32X3: return 1;  // fused: splits its operands in shared memory
    case FBST_STAGE2_DENSE_F16X3:  // the fused GEMM, after a pass for the block maxima of w unless
      return w_from_stage1 && p->tc_wmax_stage1 ? 1 : 2;  // stage 1b wrote them
    default: return 2;  // other tensor-core variants: operand preparation + GEMM
  }
}

}  // namespace fbst
