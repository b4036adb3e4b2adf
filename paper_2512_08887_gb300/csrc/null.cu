// Beamspace interference nulling (Sec. VIII-B, Eq. (14)) on top of an FBST plan.
//
// For interferer beams p_1..p_P of the plan's grid, every output beam b gets the bracket of Eq. (14),
//   wt_b = w_b - sum_j G_{b,j} w_{p_j},   G_{b,j} = F_b^H F_{p_j} (F_{p_j}^H F_{p_j} + delta I)^{-1},
// and then the plan's own stage 2: bhat_b = F_u A_b^{-1} wt_b.
//
// G_{b,j} is precomputed at plan time, as the paper's form of Eq. (14) suggests, because it is the
// well-conditioned object: applying its two factors at run time (beta_j = A_{p_j}^{-1} w_{p_j}
// first) passes through beta_j, whose components along the small eigenvectors of A_{p_j} are
// amplified by up to its condition number (~2/delta_rel), so rounding beta_j to FP32 and
// contracting it with F_b^H F_{p_j} loses about that factor in the bracket. G_{b,j} w_{p_j} has no
// such intermediate.
//
// Plan time, in FP64 with exact integer phase reduction:
//   XV64[j]   Gohberg-Semencul spectra of A_{p_j}^{-1} (from the plan's FP64 Levinson generators)
//   Gn[b][ell][j*L + k] = (F_b^H F_{p_j} A_{p_j}^{-1})[ell, k]: row ell of F_b^H F_{p_j} from its
//             closed form, times A_{p_j}^{-1} by the FP64 Gohberg-Semencul apply (Sec. V), rounded
//             to complex64 once                                        B x L x P*L complex64
// Run time, per chunk of at most max_blocks blocks:
//   k_null_gather  rhs[blk][j*L + k] = w[blk][p_j][k] (the interferers' stage-1 vectors)
//   contraction    corr[blk][b][ell] = sum_{j,k} Gn[b][ell][j*L + k] rhs[blk][j*L + k]
//                  by the FP32 CUDA-core kernel of the dense stage 2 or its split-TF32 tensor-core
//                  kernel, both reading one shared right-hand side for every beam, driven through
//                  a plan descriptor whose N is L and whose L is P*L: the contraction has the shape
//                  of the dense stage 2
//   k_null_sub     wt = w - corr
//
// The closed form of the cross Gram matrix: with [F_b]_{(m,n),ell} =
// exp(-2*pi*i*tau_{b,m}/fb) exp(i*omega_ell*(n - tau_{b,m})) (Eq. (6)),
//   (F_b^H F_p)[ell,k] = D_N(2*pi*eps*(k-ell)/L) * prod_axes sum_{m<M_axis} exp(i*theta_axis*m),
//   theta_axis = 2*pi*rho*[(u_b - u_p)/fb + eps*(ell'*u_b - k'*u_p)/L]
// with u the beam's direction cosine along that axis and D_N(x) = sum_{n<N} exp(i*x*n). For b = p it
// is the Toeplitz A_b - delta I of Sec. V; for b != p the carriers no longer cancel.
//
// The time-domain form (Eq. (15)) works on time-domain beams: out_b = y_b - sum_j G'_{b,j} y_j with
// y_j = F_x A_{p_j}^{-1} w_{p_j} the interferer's beam over a broader interval of 2L samples (F_x
// of full column rank and well conditioned there) and G'_{b,j} = F_u A_b^{-1} (F_b^H F_{p_j}) F_x^+,
// applied factor by factor at run time: F_x^+ (per interferer, FP32 CUDA cores), the contraction
// above with the cross Gram matrices in place of G_{b,j}, the plan's stage 2, and a subtraction.
// Plan time: the cross Gram rows (k_null_G without the apply); F_x A_{p_j}^{-1} (k_null_rows_gs,
// FP64 Gohberg-Semencul on the rows of F_x, kept in FP64: the interferers' beams over the broader
// interval are summed from it in FP64 by k_null_yext64); and F_x^+ = T^{-1} F_x^H with the
// Hermitian Toeplitz T = F_x^H F_x, whose Levinson column is computed on the host in FP64 and whose
// inverse is applied to the rows of F_x by the same FP64 Gohberg-Semencul kernel.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "gs.cuh"
#include "launch_util.cuh"
#include "spline.cuh"

namespace fbst {
namespace {

constexpr int kMaxInterferers = 16;

struct null_consts {
  int64_t en, ed;       // epsilon = en/ed
  int64_t fp, fq;       // fb = fp/fq; rho = fp/(2 fq + fp)
  int N, L, P;
  int mx, my, bx, by;   // element and beam grids (linear array: my = by = 1)
  int ip[kMaxInterferers];
  int offgrid;          // 1: the interferers are the directions (up, vp), not grid beams ip
  double up[kMaxInterferers], vp[kMaxInterferers];
};

// q reduced exactly modulo 2D into [-D, D).
__device__ __forceinline__ int64_t red_2D(int64_t q, int64_t D) {
  const int64_t twoD = 2 * D;
  int64_t m = q % twoD;
  if (m < 0) m += twoD;
  if (m >= D) m -= twoD;
  return m;
}

// sin(pi*q/D) and exp(i*pi*q/D) after the exact reduction of q modulo 2D, in FP64.
__device__ __forceinline__ double sinpi_red(int64_t q, int64_t D) { return sinpi((double)red_2D(q, D) / (double)D); }

__device__ __forceinline__ double2 expipi_red(int64_t q, int64_t D) {
  double s, c;
  sincospi((double)red_2D(q, D) / (double)D, &s, &c);
  return make_double2(c, s);
}

// sum_{m<count} exp(i*theta*m) with theta = pi*Y/D: count when theta = 0 mod 2*pi, else
// exp(i*theta*(count-1)/2) sin(count*theta/2) / sin(theta/2). Each factor has period 4D in Y, so
// Y is reduced modulo 4D first; the host checks that count*4D fits in 63 bits.
__device__ double2 dirichlet_d(int64_t Y, int64_t D, int count) {
  int64_t y = Y % (4 * D);
  if (y < 0) y += 4 * D;
  if (y % (2 * D) == 0) return make_double2((double)count, 0.0);
  const double q = sinpi_red((int64_t)count * y, 2 * D) / sinpi_red(y, 2 * D);
  const double2 ph = expipi_red((int64_t)(count - 1) * y, 2 * D);
  return make_double2(ph.x * q, ph.y * q);
}

// theta_axis = pi*Y/D for output grid index a and interferer grid index ap along an axis of nb
// beams: u_a = (2a - nb)/nb, rho/fb = fq/rden and rho*eps/L = fp*en/(rden*ed*L) with
// rden = 2 fq + fp give D = rden*ed*L*nb and
// Y = 2*(2*fq*(a - ap)*ed*L + fp*en*(ell'*(2a - nb) - k'*(2ap - nb))).
__device__ __forceinline__ int64_t axis_Y(const null_consts& c, int a, int ap, int nb, int64_t lp, int64_t kp) {
  return 2 * (2 * c.fq * (int64_t)(a - ap) * c.ed * c.L + c.fp * c.en * (lp * (2 * a - nb) - kp * (2 * ap - nb)));
}

// (F_b^H F_{p_j})[ell, k] in FP64 from the closed form (see the top of this file).
// sum_{m<count} exp(2*pi*i*phi*m) for a real phi (cycles) in FP64 (the element factor toward an
// off-grid direction, whose phases are not rational): exp(i*pi*phi*(count-1)) sin(pi*count*phi) /
// sin(pi*phi), or count when phi is an integer.
__device__ double2 dirichlet_phi(double phi, int count) {
  const double den = sinpi(phi);
  if (den == 0.0) return make_double2((double)count, 0.0);
  double sn, cs;
  sincospi(phi * (count - 1), &sn, &cs);
  const double q = sinpi(phi * count) / den;
  return make_double2(cs * q, sn * q);
}

__device__ __forceinline__ double2 cross_gram_entry(const null_consts& c, int b, int j, int ell, int k) {
  const int L = c.L;
  const int64_t rden = 2 * c.fq + c.fp;
  const int a = b / c.by, cy = b % c.by;
  const int64_t lp = (int64_t)ell + 1 - L / 2, kp = (int64_t)k + 1 - L / 2;
  const double2 tf = dirichlet_d(2 * c.en * (int64_t)(k - ell), c.ed * L, c.N);
  const bool two = c.my > 1 || c.by > 1;
  if (c.offgrid) {
    // theta_axis / (2 pi) = rho [(u_b - u_p)/fb + eps (ell' u_b - k' u_p)/L] in FP64.
    const double rho = (double)c.fp / (double)rden, fbv = (double)c.fp / (double)c.fq;
    const double eps = (double)c.en / (double)c.ed;
    auto phi = [&](double ub, double upj) { return rho * ((ub - upj) / fbv + eps * ((double)lp * ub - (double)kp * upj) / L); };
    double2 v = cmul(tf, dirichlet_phi(phi(-1.0 + 2.0 * a / c.bx, c.up[j]), c.mx));
    if (two) v = cmul(v, dirichlet_phi(phi(-1.0 + 2.0 * cy / c.by, c.vp[j]), c.my));
    return v;
  }
  const int pb = c.ip[j], ap = pb / c.by, cp = pb % c.by;
  double2 v = cmul(tf, dirichlet_d(axis_Y(c, a, ap, c.bx, lp, kp), rden * c.ed * L * c.bx, c.mx));
  if (two) v = cmul(v, dirichlet_d(axis_Y(c, cy, cp, c.by, lp, kp), rden * c.ed * L * c.by, c.my));
  return v;
}

// Gohberg-Semencul spectra of the interferers' A_p^{-1} (Sec. V) in FP64, before their forward FFT:
// row 2j holds x / (sqrt(x_0) P) and row 2j+1 holds Z J conj(x) / (sqrt(x_0) P), both zero-padded
// to P, with x the FP64 first column of A_{p_j}^{-1} (the plan's for a grid beam, the direction's
// own for an off-grid interferer).
__global__ void k_null_gs_rows(const double2* __restrict__ x64, double2* __restrict__ rows, null_consts c, int P,
                               int* status) {
  const int j = blockIdx.y, L = c.L;
  const double2* x = x64 + (size_t)(c.offgrid ? j : c.ip[j]) * L;   // off grid: the directions' own x
  const double x0 = x[0].x;
  if (!(x0 > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(status, (int)FBST_ERR_NUMERIC);
    return;
  }
  const double sc = 1.0 / (sqrt(x0) * P);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    rows[((size_t)j * 2 + 0) * P + k] = k < L ? cscale(x[k], sc) : make_double2(0.0, 0.0);
    rows[((size_t)j * 2 + 1) * P + k] = (k >= 1 && k < L) ? cscale(cconj(x[L - k]), sc) : make_double2(0.0, 0.0);
  }
}

template <int PG> struct gs64_e { static constexpr int value = PG >= 2048 ? 16 : (PG >= 8 ? 8 : 2); };

// Gn[b][ell][j*L + k] = (F_b^H F_{p_j} A_{p_j}^{-1})[ell, k] in FP64, rounded once. Row ell of a
// product r A^{-1} with A Hermitian is conj(A^{-1} conj(r)): the row of the cross Gram matrix is
// conjugated, taken through the FP64 Gohberg-Semencul apply of A_{p_j}^{-1} and conjugated back.
// One CTA per (ell, b, j).
// APPLY = false stores the cross Gram matrix F_b^H F_{p_j} itself (the time-domain form of Eq. (15)).
template <int PG, bool APPLY>
__global__ void __launch_bounds__(PG / gs64_e<PG>::value)
k_null_G(const double2* __restrict__ XV64, float2* __restrict__ Gn, const __grid_constant__ null_consts c,
         const double2* __restrict__ tw) {
  constexpr int E = gs64_e<PG>::value, T = PG / E;
  extern __shared__ double2 sm64[];
  const int ell = blockIdx.x, b = blockIdx.y, j = blockIdx.z, t = threadIdx.x, L = c.L, PL = c.P * c.L;
  const double2* Xj = XV64 + (size_t)j * 2 * PG;
  double2 v[E], X[E], Vv[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    v[r] = i < L ? cconj(cross_gram_entry(c, b, j, ell, i)) : make_double2(0.0, 0.0);
    X[r] = Xj[i];
    Vv[r] = Xj[PG + i];
  }
  if constexpr (APPLY) gs_apply<PG, E>(v, X, Vv, sm64, tw, t, L);
  float2* row = Gn + ((size_t)b * L + ell) * PL + (size_t)j * L;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    if (i < L) row[i] = make_float2((float)v[r].x, (float)-v[r].y);
  }
}

// Gx[j][n][k] = (R A_j^{-1})[n, k] for the FP64 rows R [nrows][L] (row n through the same
// conjugate Gohberg-Semencul apply as k_null_G, with the spectra of A_j), kept in FP64. One CTA
// per (n, j).
template <int PG>
__global__ void __launch_bounds__(PG / gs64_e<PG>::value)
k_null_rows_gs(const double2* __restrict__ XV64, const double2* __restrict__ R, double2* __restrict__ Gx, int L,
               int nrows, const double2* __restrict__ tw) {
  constexpr int E = gs64_e<PG>::value, T = PG / E;
  extern __shared__ double2 sm64[];
  const int n = blockIdx.x, j = blockIdx.z, t = threadIdx.x;
  const double2* Xj = XV64 + (size_t)j * 2 * PG;
  double2 v[E], X[E], Vv[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    v[r] = i < L ? cconj(R[(size_t)n * L + i]) : make_double2(0.0, 0.0);
    X[r] = Xj[i];
    Vv[r] = Xj[PG + i];
  }
  gs_apply<PG, E>(v, X, Vv, sm64, tw, t, L);
  double2* row = Gx + ((size_t)j * nrows + n) * L;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    if (i < L) row[i] = cconj(v[r]);
  }
}

// The interferers' beams over the broader interval, yext[blk][j][n] = sum_k Gx[j][n][k] w[blk][p_j][k],
// accumulated in FP64 and rounded once: Gx = F_x A_{p_j}^{-1} has entries of the size of
// ||A^{-1}|| whose products cancel down to the much smaller beam, so an FP32 sum would lose that
// factor. One warp per (n, j) and 8 blocks; lanes split k, then a warp sum.
__global__ void k_null_yext64(const double2* __restrict__ Gx, const float2* __restrict__ w, float2* __restrict__ yext,
                              const __grid_constant__ null_consts c, int B, int nb, int Nu) {
  constexpr int KB = 8;
  const int n = blockIdx.x, j = blockIdx.y, blk0 = blockIdx.z * KB, lane = threadIdx.x, L = c.L;
  const double2* g = Gx + ((size_t)j * Nu + n) * L;
  double2 acc[KB];
#pragma unroll
  for (int q = 0; q < KB; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int k = lane; k < L; k += 32) {
    const double2 gk = g[k];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      if (blk0 + q < nb) {
        const float2 x = w[((size_t)(blk0 + q) * B + c.ip[j]) * L + k];
        acc[q].x += gk.x * x.x - gk.y * x.y;
        acc[q].y += gk.x * x.y + gk.y * x.x;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < KB; ++q) {
    double re = acc[q].x, im = acc[q].y;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0 && blk0 + q < nb) yext[((size_t)(blk0 + q) * c.P + j) * Nu + n] = make_float2((float)re, (float)im);
  }
}

template <int PG>
int build_G_P(const double2* XV64, float2* Gn, const null_consts& c, int B, const double2* tw, bool apply,
              const double2* rows, int nrows, double2* Gx, cudaStream_t s) {
  constexpr int E = gs64_e<PG>::value;
  const size_t smem = 2 * sizeof(double2) * fft_smem_elems<double2>(PG);
  if (rows) {
    FBST_CUDA_TRY(cudaFuncSetAttribute(k_null_rows_gs<PG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_null_rows_gs<PG><<<dim3(nrows, 1, c.P), PG / E, smem, s>>>(XV64, rows, Gx, c.L, nrows, tw);
  } else if (apply) {
    FBST_CUDA_TRY(cudaFuncSetAttribute(k_null_G<PG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_null_G<PG, true><<<dim3(c.L, B, c.P), PG / E, smem, s>>>(XV64, Gn, c, tw);
  } else {
    FBST_CUDA_TRY(cudaFuncSetAttribute(k_null_G<PG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_null_G<PG, false><<<dim3(c.L, B, c.P), PG / E, smem, s>>>(XV64, Gn, c, tw);
  }
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// Eq. (14)'s G_{b,j} (apply), the cross Gram matrices alone (!apply), or with `rows` the FP64
// products rows x A_j^{-1} (nrows rows, c.P matrices A_j given by the spectra XV64) into Gx.
int build_G(int PG, const double2* XV64, float2* Gn, const null_consts& c, int B, const double2* tw, cudaStream_t s,
            bool apply = true, const double2* rows = nullptr, int nrows = 0, double2* Gx = nullptr) {
  switch (PG) {
    case 16: return build_G_P<16>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 32: return build_G_P<32>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 64: return build_G_P<64>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 128: return build_G_P<128>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 256: return build_G_P<256>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 512: return build_G_P<512>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 1024: return build_G_P<1024>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 2048: return build_G_P<2048>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    case 4096: return build_G_P<4096>(XV64, Gn, c, B, tw, apply, rows, nrows, Gx, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

// The contraction's right-hand side: rhs[blk][cp][j*L + k] = w[blk][p_j][k] for cp < copies (1 for
// the tensor-core contraction, which reads one right-hand side for all beams; B for the CUDA-core
// one, which reads one per beam), as float4 pairs of complex values (L is even).
__global__ void k_null_gather(const float4* __restrict__ w, float4* __restrict__ rhs, const __grid_constant__ null_consts c,
                              int B, int copies, int nb) {
  const int L2 = c.L / 2, PL2 = c.P * L2;
  const long long total = (long long)nb * copies * PL2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % PL2);
    const long long bc = i / PL2;
    const int blk = (int)(bc / copies);
    const int j = e / L2, k = e - j * L2;
    rhs[i] = w[((size_t)blk * B + c.ip[j]) * L2 + k];
  }
}

// Off-grid interferers: rhs[blk][cp][j*L + k] = sum_{i, jj} cx_j[i] cy_j[jj] w[blk][(fx_j + i)*by + fy_j + jj][k],
// the interferer's vector interpolated from the grid beam vectors (Sec. VIII-A), float4 pairs.
__global__ void k_null_interp_rhs(const float4* __restrict__ w, float4* __restrict__ rhs,
                                  const __grid_constant__ null_consts c, const int2* __restrict__ first,
                                  const float* __restrict__ wts, int B, int copies, int nb, int Kx, int Ky) {
  const int L2 = c.L / 2, PL2 = c.P * L2;
  const long long total = (long long)nb * copies * PL2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % PL2);
    const int blk = (int)(i / PL2 / copies);
    const int j = e / L2, k = e - j * L2;
    const int2 f0 = first[j];
    const float* cx = wts + (size_t)j * (Kx + Ky);
    const float* cy = cx + Kx;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int a = 0; a < Kx; ++a)
      for (int q = 0; q < Ky; ++q) {
        const float cw = cx[a] * cy[q];
        const float4 v = w[((size_t)blk * B + (size_t)(f0.x + a) * c.by + f0.y + q) * L2 + k];
        acc.x = fmaf(cw, v.x, acc.x);
        acc.y = fmaf(cw, v.y, acc.y);
        acc.z = fmaf(cw, v.z, acc.z);
        acc.w = fmaf(cw, v.w, acc.w);
      }
    rhs[i] = acc;
  }
}

// wt = w - corr over n4 float4 (two complex values each); wt may be w.
__global__ void k_null_sub(const float4* w, const float4* __restrict__ corr, float4* wt, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
    const float4 a = w[i], b = corr[i];
    wt[i] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
  }
}

int stream_grid(long long items, int threads) {
  return (int)std::max<long long>(1, std::min<long long>((items + threads - 1) / threads, (long long)sm_count() * 8));
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

// Time-domain form (Eq. (15)): F_x[n][ell] = exp(i*omega_ell*t_n) on the broader interval of
// Nu = 2L samples t_n = n0 + n, n0 = -(2L - N)/2, in FP64 on the host, the phase eps*ell'*t/L
// reduced exactly (2*en*ell'*t modulo 2*ed*L in units of pi/(ed*L)). Twice the basis size keeps
// F_x well conditioned (its frequencies span 1.01 cycles per sample and interleave near half a
// cycle, which an interval of L samples cannot resolve).
void time_rows(const fbst_info& in, std::vector<std::complex<double>>& F) {
  const int L = in.L, Nu = 2 * L, n0 = -(Nu - in.N) / 2;
  const int64_t D = in.eps_den * (int64_t)L;
  F.assign((size_t)Nu * L, {0.0, 0.0});
  for (int n = 0; n < Nu; ++n)
    for (int ell = 0; ell < L; ++ell) {
      const int64_t lp = (int64_t)ell + 1 - L / 2, t = (int64_t)n0 + n;
      int64_t q = (2 * in.eps_num * lp * t) % (2 * D);
      if (q < 0) q += 2 * D;
      const double ang = M_PI * (double)q / (double)D;
      F[(size_t)n * L + ell] = {std::cos(ang), std::sin(ang)};
    }
}

// First row a(d) = sum_n exp(2*pi*i*eps*d*t_n/L), d < L, of the Gram matrix T = F_x^H F_x
// (Hermitian Toeplitz, T[l][k] = a(k - l)), as an FP64 direct sum with the same exact reduction.
void time_gram_row(const fbst_info& in, std::vector<std::complex<double>>& a) {
  const int L = in.L, Nu = 2 * L, n0 = -(Nu - in.N) / 2;
  const int64_t D = in.eps_den * (int64_t)L;
  a.assign(L, {0.0, 0.0});
  for (int d = 0; d < L; ++d) {
    std::complex<double> acc = 0.0;
    for (int n = 0; n < Nu; ++n) {
      int64_t q = (2 * in.eps_num * (int64_t)d * ((int64_t)n0 + n)) % (2 * D);
      if (q < 0) q += 2 * D;
      const double ang = M_PI * (double)q / (double)D;
      acc += std::complex<double>(std::cos(ang), std::sin(ang));
    }
    a[d] = acc;
  }
}

// x = T^{-1} e_0 for the Hermitian positive definite Toeplitz T with first row a, by the Levinson
// recursion in FP64 (first column c[d] = conj(a(d)); f_k solves T_k f_k = e_0 and extends as
// f_{k+1}[i] = (f_k[i] - e_k conj(f_k[k-i])) / (1 - |e_k|^2), e_k = sum_{i<k} c[k-i] f_k[i]).
bool levinson_host(const std::vector<std::complex<double>>& a, std::vector<std::complex<double>>& f) {
  const int L = (int)a.size();
  if (!(a[0].real() > 0.0)) return false;
  f.assign(L, {0.0, 0.0});
  f[0] = 1.0 / std::conj(a[0]);
  std::vector<std::complex<double>> g(L);
  for (int k = 1; k < L; ++k) {
    std::complex<double> e = 0.0;
    for (int i = 0; i < k; ++i) e += std::conj(a[k - i]) * f[i];
    const double den = 1.0 - std::norm(e);
    if (!(den > 0.0)) return false;
    for (int i = 0; i <= k; ++i) g[i] = (f[i] - e * std::conj(f[k - i])) / den;
    for (int i = 0; i <= k; ++i) f[i] = g[i];
  }
  return true;
}

}  // namespace
}  // namespace fbst

using namespace fbst;

struct fbst_null_s {
  fbst_plan_s* plan;     // the plan whose grid, workspace and stage 2 are used (not owned)
  int P;
  int contraction;       // FBST_NULL_TF32X3 or FBST_NULL_FP32
  fbst_plan_s shadow;    // descriptor of the G contraction for the dense stage-2 kernels
  float2* Q;             // Gn [B][L][P*L] complex64; freed once the tensor-core planes are built
  double2* XV64;         // [P][2][P_gs] Gohberg-Semencul spectra of the interferers, FP64
  float2* rhs;           // [max_blocks][1 or B][P*L] (one copy for the tensor-core contraction)
  float2* corr;          // [max_blocks][B][L]
  null_consts c;
  // Off-grid interferers: interpolation windows and weights of each interferer's vector.
  int Kx, Ky;
  int2* ifirst;          // [P]
  float* iwts;           // [P][Kx + Ky]
  // Time-domain form (Eq. (15)); then Q holds the cross Gram matrices F_b^H F_{p_j} themselves.
  int time_form;
  fbst_plan_s shx;       // descriptor of the per-interferer products F_x^+ y_j (B := P, N := L, L := 2L)
  double2* Gx;           // [P][2L][L] F_x A_{p_j}^{-1} (FP64): an interferer's beam over the broader interval
  float2* Xrep;          // [P][L][2L] F_x^+ = (F_x^H F_x)^{-1} F_x^H, once per interferer
  float2* yext;          // [max_blocks][P][2L] interferer beams over the broader interval
  float2* bh;            // [max_blocks][P][L] F_x^{-1} yext
  float2* tmp;           // [max_blocks][B][N] the correction in the time domain
};

// The object's blocks go back through the plan's allocator (they are in the plan's registry).
static void free_null(fbst_null_s* n) {
  void* ptrs[] = {n->Q, n->shadow.Gtc, n->XV64, n->rhs, n->corr, n->ifirst, n->iwts, n->Gx, n->Xrep, n->yext,
                  n->bh, n->tmp};
  for (void* q : ptrs) plan_free(n->plan, q);
}

// One chunk (nb <= max_blocks) of the bracket of Eq. (14): w [nb][B][L] -> wt (may be w).
static int null_chunk(fbst_null_s* n, const float2* w, float2* wt, int nb, cudaStream_t s) {
  const fbst_info& in = n->plan->info;
  const int L = in.L, B = in.B;
  const bool tc = n->contraction == FBST_NULL_TF32X3;
  {
    // One right-hand side per block, read by every beam's tile of the contraction.
    const long long n4 = (long long)nb * n->P * L / 2;
    if (n->c.offgrid)
      k_null_interp_rhs<<<stream_grid(n4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(w),
                                                             reinterpret_cast<float4*>(n->rhs), n->c, n->ifirst,
                                                             n->iwts, B, 1, nb, n->Kx, n->Ky);
    else
      k_null_gather<<<stream_grid(n4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(w),
                                                         reinterpret_cast<float4*>(n->rhs), n->c, B, 1, nb);
    FBST_CUDA_TRY(cudaGetLastError());
  }
  n->shadow.wait_ns = n->plan->wait_ns;   // the plan's wait limit applies to the contraction too
  const int r = tc ? launch_dense_tc_shared_rhs(&n->shadow, n->rhs, n->corr, nb, s)
                   : launch_dense_fp32_rhs(&n->shadow, n->rhs, n->corr, nb, true, s);
  if (r != FBST_OK) return r;
  const long long n4 = (long long)nb * B * L / 2;
  k_null_sub<<<stream_grid(n4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(w),
                                                  reinterpret_cast<const float4*>(n->corr),
                                                  reinterpret_cast<float4*>(wt), n4);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// One chunk of Eq. (15) on time-domain beams: out = y - sum_j G'_{b,j} yext_j with
// G'_{b,j} = F_u A_b^{-1} (F_b^H F_{p_j}) F_x^{-1}, applied factor by factor: bh_j = F_x^{-1} yext_j,
// corr_b = sum_j (F_b^H F_{p_j}) bh_j (the contraction of Eq. (14)'s shape with the cross Gram
// matrices), tmp = the plan's stage 2 of corr, out = y - tmp. y [nb][B][N], yext [nb][P][L]; out may
// be y.
static int time_chunk(fbst_null_s* n, const float2* y, const float2* yext, float2* out, int nb, cudaStream_t s) {
  fbst_plan_s* p = n->plan;
  const fbst_info& in = p->info;
  n->shx.G = n->Xrep;
  FBST_TRY(launch_dense_fp32_rhs(&n->shx, yext, n->bh, nb, false, s));
  n->shadow.wait_ns = p->wait_ns;
  FBST_TRY(n->contraction == FBST_NULL_TF32X3 ? launch_dense_tc_shared_rhs(&n->shadow, n->bh, n->corr, nb, s)
                                              : launch_dense_fp32_rhs(&n->shadow, n->bh, n->corr, nb, true, s));
  FBST_TRY(run_stage2(p, n->corr, n->tmp, nb, s));
  const long long n4 = (long long)nb * in.B * in.N / 2;
  k_null_sub<<<stream_grid(n4, 256), 256, 0, s>>>(reinterpret_cast<const float4*>(y),
                                                  reinterpret_cast<const float4*>(n->tmp),
                                                  reinterpret_cast<float4*>(out), n4);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// The nulling object of P interferers: grid beams `interferers`, or directions `dirs` ([P][2]
// direction cosines, interpolated from K grid beams per axis) when interferers is null.
static int null_create(fbst_null_t* out, fbst_plan_s* p, const int* interferers, const double* dirs, int K, int P,
                       int contraction, void* stream, bool time_form = false) {
  if (!out) return FBST_ERR_INVALID;
  *out = nullptr;
  if (!p || (!interferers && !dirs) || P < 1 || P > kMaxInterferers) return FBST_ERR_INVALID;
  if (contraction != FBST_NULL_TF32X3 && contraction != FBST_NULL_FP32) return FBST_ERR_INVALID;
  if (p->nu_nf) return FBST_ERR_UNSUPPORTED;   // the cross Gram closed form needs grid positions
  const fbst_info& in = p->info;
  const int L = in.L, B = in.B;
  const bool ura = p->geom.kind == FBST_URA;
  if (interferers) {
    for (int j = 0; j < P; ++j) {
      if (interferers[j] < 0 || interferers[j] >= B) return FBST_ERR_INVALID;
      for (int i = 0; i < j; ++i)
        if (interferers[i] == interferers[j]) return FBST_ERR_INVALID;
    }
  } else {
    if (K < 2 || K > kMaxWindow) return FBST_ERR_INVALID;
    for (int j = 0; j < P; ++j) {
      const double u = dirs[2 * j], v = dirs[2 * j + 1];
      if (!std::isfinite(u) || !std::isfinite(v) || std::fabs(u) > 1.0 || std::fabs(v) > 1.0) return FBST_ERR_INVALID;
      if (!ura && v != 0.0) return FBST_ERR_INVALID;
    }
    int cur = -1;
    FBST_CUDA_TRY(cudaGetDevice(&cur));
    if (cur != p->device) return FBST_ERR_INVALID;
  }
  // 64-bit headroom of the exact phase reductions: |Y| and count * 4D of every Dirichlet sum.
  {
    const long double lim = std::ldexp(1.0L, 62);
    const long double rden = 2.0L * in.fb_den + in.fb_num;
    const int ax_n[2] = {p->geom.bx, p->geom.by}, ax_m[2] = {p->geom.mx, p->geom.my};
    for (int a = 0; a < 2; ++a) {
      const long double D = rden * in.eps_den * L * ax_n[a];
      const long double Y = 2.0L * (2.0L * in.fb_den * ax_n[a] * in.eps_den * L +
                                    (long double)in.fb_num * in.eps_num * (L / 2 + 1) * 2.0L * ax_n[a]);
      if (Y >= lim || 4.0L * D * ax_m[a] >= lim) return FBST_ERR_UNSUPPORTED;
    }
    if (4.0L * in.eps_den * L * in.N >= lim) return FBST_ERR_UNSUPPORTED;
  }
  if (contraction == FBST_NULL_TF32X3 && ((size_t)P * L) % 8 != 0) return FBST_ERR_UNSUPPORTED;
  // Time-domain form: grid interferers, an interval of 2L samples centred on the block (N even:
  // the interval's start is an integer and the subtraction runs on complex pairs), L <= 1024.
  if (time_form && (!interferers || in.N % 2 != 0 || L > 1024)) return FBST_ERR_UNSUPPORTED;

  fbst_null_s* n = new (std::nothrow) fbst_null_s();
  if (!n) return FBST_ERR_OOM;
  std::memset(n, 0, sizeof(*n));
  n->plan = p;
  n->P = P;
  n->contraction = contraction;
  n->time_form = time_form ? 1 : 0;
  null_consts& c = n->c;
  c.en = in.eps_num;
  c.ed = in.eps_den;
  c.fp = in.fb_num;
  c.fq = in.fb_den;
  c.N = in.N;
  c.L = L;
  c.P = P;
  c.mx = p->geom.mx;
  c.my = p->geom.my;
  c.bx = p->geom.bx;
  c.by = p->geom.by;
  c.offgrid = interferers ? 0 : 1;
  std::vector<int2> ifirst;
  std::vector<float> iwts;
  for (int j = 0; j < P; ++j) {
    if (interferers) {
      c.ip[j] = interferers[j];
    } else {
      c.up[j] = dirs[2 * j];
      c.vp[j] = dirs[2 * j + 1];
    }
  }
  if (!interferers) {
    n->Kx = std::min(K, p->geom.bx);
    n->Ky = ura ? std::min(K, p->geom.by) : 1;
    ifirst.resize(P);
    iwts.resize((size_t)P * (n->Kx + n->Ky));
    for (int j = 0; j < P; ++j) {
      int fx = 0, fy = 0;
      interp_terms(p->geom.bx, p->geom.by, ura, dirs[2 * j], dirs[2 * j + 1], n->Kx, n->Ky, &fx, &fy,
                   &iwts[(size_t)j * (n->Kx + n->Ky)]);
      ifirst[j] = make_int2(fx, fy);
    }
  }

  // The contraction's descriptor: the dense stage-2 kernels with N := L and L := P*L.
  fbst_plan_s& sh = n->shadow;
  sh.info = in;
  sh.info.N = L;
  sh.info.L = P * L;
  sh.info.stage2 = contraction == FBST_NULL_TF32X3 ? FBST_STAGE2_DENSE_TF32X3 : FBST_STAGE2_DENSE_FP32;
  sh.geom = p->geom;
  sh.band = p->band;
  sh.device = p->device;
  sh.d_status = p->d_status;
  share_allocator(&sh, p);

  // The per-interferer L x L products of the time-domain form: the dense FP32 kernel with B := P.
  if (time_form) {
    fbst_plan_s& sx = n->shx;
    sx.info = in;
    sx.info.B = P;
    sx.info.N = L;
    sx.info.L = 2 * L;
    sx.info.stage2 = FBST_STAGE2_DENSE_FP32;
    sx.geom = p->geom;
    sx.band = p->band;
    sx.device = p->device;
    sx.d_status = p->d_status;
    share_allocator(&sx, p);
  }

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int maxb = p->band.max_blocks;
  double* dirs_dev = nullptr;
  double2* xdir = nullptr;
  double2* rows64 = nullptr;   // F_x (FP64), time-domain form
  double2* xvt = nullptr;      // Gohberg-Semencul spectra of T = F_x^H F_x
  double2* xht = nullptr;      // F_x T^{-1} = (F_x^+)^H (FP64)
  int r = FBST_OK;
  do {
    if ((r = plan_alloc_n(p, &n->Q, (size_t)B * L * P * L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &n->XV64, (size_t)P * 2 * in.P_gs)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &n->rhs, (size_t)maxb * P * L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &n->corr, (size_t)maxb * B * L)) != FBST_OK) break;
    if (time_form) {
      if ((r = plan_alloc_n(p, &n->Gx, (size_t)P * 2 * L * L)) != FBST_OK) break;   // FP64
      if ((r = plan_alloc_n(p, &n->Xrep, (size_t)P * L * 2 * L)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &n->yext, (size_t)maxb * P * 2 * L)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &n->bh, (size_t)maxb * P * L)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &n->tmp, (size_t)maxb * B * in.N)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &rows64, (size_t)2 * L * L)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &xvt, (size_t)2 * in.P_gs)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &xht, (size_t)2 * L * L)) != FBST_OK) break;
    }
    if (!interferers) {
      if ((r = plan_alloc_n(p, &n->ifirst, (size_t)P)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &n->iwts, iwts.size())) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &dirs_dev, 2 * (size_t)P)) != FBST_OK) break;
      if ((r = plan_alloc_n(p, &xdir, (size_t)P * L)) != FBST_OK) break;
    }
    // Allocated in stream order on the plan's stream: make the blocks usable on `s`.
    if (cudaStreamSynchronize(p->mem_stream) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    const double2* xsrc = p->x64;
    if (!interferers) {
      if (cudaMemcpy(n->ifirst, ifirst.data(), sizeof(int2) * P, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(n->iwts, iwts.data(), sizeof(float) * iwts.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(dirs_dev, dirs, sizeof(double) * 2 * P, cudaMemcpyHostToDevice) != cudaSuccess) {
        r = FBST_ERR_CUDA;
        break;
      }
      if ((r = build_direction_x(p, dirs_dev, P, xdir, s)) != FBST_OK) break;
      xsrc = xdir;
    }
    k_null_gs_rows<<<dim3(std::min((in.P_gs + 255) / 256, 16), P), 256, 0, s>>>(xsrc, n->XV64, c, in.P_gs,
                                                                                p->d_status);
    if (cudaGetLastError() != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    if ((r = fft64_rows(n->XV64, 2 * P, in.P_gs, p->tw64, -1, s)) != FBST_OK) break;
    if ((r = build_G(in.P_gs, n->XV64, n->Q, c, B, p->tw64, s, !time_form)) != FBST_OK) break;
    if (time_form) {
      // F_x (FP64, host) -> Gx = F_x A_{p_j}^{-1} and F_x T^{-1} = (F_x^+)^H, T = F_x^H F_x, both
      // by the FP64 Gohberg-Semencul apply on the rows of F_x (T's spectra from its Levinson
      // column, computed on the host); F_x^+ rounded once to complex64.
      const int Nu = 2 * L, PG = in.P_gs;
      std::vector<std::complex<double>> F, a, xT;
      time_rows(in, F);
      time_gram_row(in, a);
      if (!levinson_host(a, xT) || !(xT[0].real() > 0.0)) { r = FBST_ERR_NUMERIC; break; }
      std::vector<std::complex<double>> sp((size_t)2 * PG, {0.0, 0.0});
      const double sc = 1.0 / (std::sqrt(xT[0].real()) * PG);
      for (int k = 0; k < L; ++k) {
        sp[k] = xT[k] * sc;
        if (k >= 1) sp[PG + k] = std::conj(xT[L - k]) * sc;
      }
      if (cudaMemcpy(rows64, F.data(), sizeof(double2) * F.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(xvt, sp.data(), sizeof(double2) * sp.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        r = FBST_ERR_CUDA;
        break;
      }
      if ((r = fft64_rows(xvt, 2, PG, p->tw64, -1, s)) != FBST_OK) break;
      if ((r = build_G(PG, n->XV64, nullptr, c, B, p->tw64, s, true, rows64, Nu, n->Gx)) != FBST_OK) break;
      null_consts c1 = c;
      c1.P = 1;
      if ((r = build_G(PG, xvt, nullptr, c1, B, p->tw64, s, true, rows64, Nu, xht)) != FBST_OK) break;
      std::vector<std::complex<double>> xh((size_t)Nu * L);
      if (cudaMemcpyAsync(xh.data(), xht, sizeof(double2) * xh.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        r = FBST_ERR_CUDA;
        break;
      }
      // F_x^+ [L][Nu] = conj(xh)^T, once per interferer.
      std::vector<float2> xi((size_t)P * L * Nu);
      for (int ell = 0; ell < L; ++ell)
        for (int nn = 0; nn < Nu; ++nn) {
          const std::complex<double> v = std::conj(xh[(size_t)nn * L + ell]);
          for (int j = 0; j < P; ++j)
            xi[((size_t)j * L + ell) * Nu + nn] = make_float2((float)v.real(), (float)v.imag());
        }
      if (cudaMemcpy(n->Xrep, xi.data(), sizeof(float2) * xi.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        r = FBST_ERR_CUDA;
        break;
      }
    }
    sh.G = n->Q;
    if (contraction == FBST_NULL_TF32X3) {
      if ((r = build_dense_tc_operand(&sh, s)) != FBST_OK) break;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    int st = 0;
    if (cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    if (st != 0) {
      cudaMemset(p->d_status, 0, sizeof(int));
      r = st;
      break;
    }
    if (contraction == FBST_NULL_TF32X3) {
      plan_free(p, n->Q);
      n->Q = nullptr;
      sh.G = nullptr;
    }
  } while (0);
  cudaStreamSynchronize(s);
  plan_free(p, dirs_dev);
  plan_free(p, xdir);
  plan_free(p, rows64);
  plan_free(p, xvt);
  plan_free(p, xht);
  if (r != FBST_OK) {
    free_null(n);
    delete n;
    return r;
  }
  *out = n;
  return FBST_OK;
}

extern "C" {

int fbst_null_create(fbst_null_t* out, fbst_plan_t p, const int* interferers, int P, int contraction, void* stream) {
  if (out) *out = nullptr;
  if (!interferers) return FBST_ERR_INVALID;
  return null_create(out, p, interferers, nullptr, 0, P, contraction, stream);
}

int fbst_null_create_directions(fbst_null_t* out, fbst_plan_t p, const double* directions, int P, int K,
                                int contraction, void* stream) {
  if (out) *out = nullptr;
  if (!directions) return FBST_ERR_INVALID;
  return null_create(out, p, nullptr, directions, K, P, contraction, stream);
}

int fbst_null_create_time(fbst_null_t* out, fbst_plan_t p, const int* interferers, int P, int contraction,
                          void* stream) {
  if (out) *out = nullptr;
  if (!interferers) return FBST_ERR_INVALID;
  return null_create(out, p, interferers, nullptr, 0, P, contraction, stream, true);
}

int fbst_null_apply_time(fbst_null_t n, const void* y, const void* y_int, void* out, int nblk, void* stream) {
  if (!n || nblk < 0) return FBST_ERR_INVALID;
  if (!n->time_form) return FBST_ERR_UNSUPPORTED;
  if (nblk == 0) return FBST_OK;
  if (!y || !y_int || !out || !aligned16(y) || !aligned16(y_int) || !aligned16(out)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = n->plan->info;
  const int maxb = n->plan->band.max_blocks;
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    const size_t oy = (size_t)c0 * in.B * in.N, oi = (size_t)c0 * n->P * 2 * in.L;
    FBST_TRY(time_chunk(n, static_cast<const float2*>(y) + oy, static_cast<const float2*>(y_int) + oi,
                        static_cast<float2*>(out) + oy, nb, s));
  }
  return FBST_OK;
}

int fbst_null_apply(fbst_null_t n, const void* w, void* wt, int nblk, void* stream) {
  if (!n || nblk < 0) return FBST_ERR_INVALID;
  if (n->time_form) return FBST_ERR_UNSUPPORTED;
  if (nblk == 0) return FBST_OK;
  if (!w || !wt || !aligned16(w) || !aligned16(wt)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fbst_info& in = n->plan->info;
  const int maxb = n->plan->band.max_blocks;
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    const size_t off = (size_t)c0 * in.B * in.L;
    FBST_TRY(null_chunk(n, static_cast<const float2*>(w) + off, static_cast<float2*>(wt) + off, nb, s));
  }
  return FBST_OK;
}

int fbst_null_execute(fbst_null_t n, const void* y, void* bhat, int nblk, void* stream) {
  if (!n || nblk < 0) return FBST_ERR_INVALID;
  if (nblk == 0) return FBST_OK;
  if (!y || !bhat || !aligned16(y) || !aligned16(bhat)) return FBST_ERR_INVALID;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fbst_plan_s* p = n->plan;
  const fbst_info& in = p->info;
  const int maxb = p->band.max_blocks;
  for (int c0 = 0; c0 < nblk; c0 += maxb) {
    const int nb = std::min(maxb, nblk - c0);
    float2* ob = static_cast<float2*>(bhat) + (size_t)c0 * in.B * in.N;
    FBST_TRY(launch_czt_time(p, static_cast<const float2*>(y) + (size_t)c0 * in.M * in.N, p->ws_yhat, nb, s));
    if (n->time_form) {
      // Eq. (15): the plain beams, the interferers' beams over the broader interval, then the
      // time-domain subtraction.
      FBST_TRY(launch_czt_space_scaled(p, p->ws_yhat, p->ws_w, nb, 0, s));
      FBST_TRY(run_stage2(p, p->ws_w, ob, nb, s, true));
      k_null_yext64<<<dim3(2 * in.L, n->P, (nb + 7) / 8), 32, 0, s>>>(n->Gx, p->ws_w, n->yext, n->c, in.B, nb,
                                                                       2 * in.L);
      FBST_CUDA_TRY(cudaGetLastError());
      FBST_TRY(time_chunk(n, ob, n->yext, ob, nb, s));
      continue;
    }
    FBST_TRY(launch_czt_space(p, p->ws_yhat, p->ws_w, nb, s));
    FBST_TRY(null_chunk(n, p->ws_w, p->ws_w, nb, s));
    FBST_TRY(run_stage2(p, p->ws_w, ob, nb, s));
  }
  return FBST_OK;
}

int fbst_null_launch_count(fbst_null_t n, int nblk) {
  if (!n || nblk <= 0) return 0;
  const int maxb = n->plan->band.max_blocks;
  const int chunks = (nblk + maxb - 1) / maxb;
  if (n->time_form)  // stage 1, plain stage 2, F_x A_p^{-1} (FP64), F_x^{-1}, contraction, stage 2, sub
    return chunks * (2 + stage2_launches(n->plan, true) + 4 + stage2_launches(n->plan, false));
  return chunks * (2 + 3 + stage2_launches(n->plan, false));
}

int fbst_null_destroy(fbst_null_t n) {
  if (!n) return FBST_OK;
  free_null(n);
  delete n;
  return FBST_OK;
}

}  // extern "C"
