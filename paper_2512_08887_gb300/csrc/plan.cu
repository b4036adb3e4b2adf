// Plan construction: parameter derivation (host) and the plan-time tables (GPU, FP64 + int64).
//
// Every quadratic chirp phase of the method has the form pi * q / D with integer q and D once
// epsilon and the fractional bandwidth are taken as fractions (Eq. (3), Eq. (12), Sec. IV):
// the plan reduces q modulo 2D exactly in 64-bit integers and only then evaluates sincospi in
// FP64, so no table entry carries the O(n^2 * ulp) phase error a floating-point product would.
// The Toeplitz generators of Sec. V are closed-form Dirichlet kernels evaluated the same way,
// the first column of each A_b^{-1} comes from an FP64 Levinson recursion, and the
// Gohberg-Semencul spectra / dense operators are built from it in FP64 and rounded once.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "common.cuh"
#include "fft.cuh"
#include "gs.cuh"

namespace fbst {

// ---------------------------------------------------------------------------------------------
// Host-side derivation
// ---------------------------------------------------------------------------------------------
static int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Nearest fraction num/den to x with 1 <= den <= maxden (smallest den on ties).
static void rationalize(double x, int64_t maxden, int64_t* num, int64_t* den) {
  double best = INFINITY;
  int64_t bn = 0, bd = 1;
  for (int64_t d = 1; d <= maxden; ++d) {
    const double n = std::nearbyint(x * (double)d);
    const double err = std::fabs(x - n / (double)d);
    if (err < best) {
      best = err;
      bn = (int64_t)n;
      bd = d;
      if (err == 0.0) break;
    }
  }
  const int64_t g = gcd64(bn, bd);
  *num = bn / (g ? g : 1);
  *den = bd / (g ? g : 1);
}

static int pow2_at_least(int64_t n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

static int ilog2(int p) {
  int l = 0;
  while ((1 << l) < p) ++l;
  return l;
}

constexpr int kMinFFT = 16;
constexpr int64_t kMaxDen = 1000;

}  // namespace fbst

using namespace fbst;

extern "C" int fbst_derive(const fbst_geometry* g, int M, int N, int B, const fbst_band* band,
                           fbst_info* out) {
  if (!g || !band || !out) return FBST_ERR_INVALID;
  std::memset(out, 0, sizeof(*out));
  if (g->kind != FBST_ULA && g->kind != FBST_URA) return FBST_ERR_INVALID;
  if (g->mx < 1 || g->my < 1 || g->bx < 1 || g->by < 1) return FBST_ERR_INVALID;
  if (g->kind == FBST_ULA && (g->my != 1 || g->by != 1)) return FBST_ERR_INVALID;
  if ((int64_t)g->mx * g->my != M || (int64_t)g->bx * g->by != B) return FBST_ERR_INVALID;
  if (N < 1 || M < 1 || B < 1) return FBST_ERR_INVALID;
  if (band->gamma_num < 1 || band->gamma_den < 1) return FBST_ERR_INVALID;
  if (((int64_t)N * band->gamma_num) % band->gamma_den != 0) return FBST_ERR_INVALID;
  const int64_t L64 = (int64_t)N * band->gamma_num / band->gamma_den;
  if (L64 < 2 || (L64 & 1) || L64 < N) return FBST_ERR_INVALID;
  if (!(band->frac_bw > 0.0 && band->frac_bw < 2.0)) return FBST_ERR_INVALID;
  if (!(band->epsilon >= 1.0 && band->epsilon <= 2.0)) return FBST_ERR_INVALID;
  if (!(band->delta > 0.0) || !std::isfinite(band->delta)) return FBST_ERR_INVALID;
  if (band->max_blocks < 1) return FBST_ERR_INVALID;
  if (band->generator_solver != FBST_GEN_LEVINSON && band->generator_solver != FBST_GEN_SUPERFAST)
    return FBST_ERR_INVALID;
  switch (band->stage2) {
    case FBST_STAGE2_AUTO: case FBST_STAGE2_GS: case FBST_STAGE2_GS_IR1: case FBST_STAGE2_DENSE_FP32:
    case FBST_STAGE2_DENSE_BF16X3: case FBST_STAGE2_DENSE_TF32: case FBST_STAGE2_DENSE_TF32X3:
    case FBST_STAGE2_DENSE_F16X3: break;
    default: return FBST_ERR_INVALID;
  }
  const int L = (int)L64;
  out->M = M;
  out->N = N;
  out->B = B;
  out->L = L;

  rationalize(band->epsilon, kMaxDen, &out->eps_num, &out->eps_den);
  rationalize(band->frac_bw, kMaxDen, &out->fb_num, &out->fb_den);
  if (out->fb_num < 1 || out->fb_num >= 2 * out->fb_den || out->eps_num < out->eps_den)
    return FBST_ERR_INVALID;
  const double fb = (double)out->fb_num / (double)out->fb_den;
  out->rho = fb / (2.0 + fb);
  out->delta = band->delta_relative ? band->delta * (double)M * (double)N : band->delta;

  // Stage 1a: one forward transform and S inverse transforms of size pow2(N + L/S - 1).
  {
    const int P1 = std::max(kMinFFT, pow2_at_least((int64_t)N + L - 1));
    const int P2 = std::max(kMinFFT, pow2_at_least((int64_t)N + L / 2 - 1));
    const double c1 = 2.0 * P1 * ilog2(P1), c2 = 3.0 * P2 * ilog2(P2);
    if (c2 < c1) { out->P_time = P2; out->S_time = 2; } else { out->P_time = P1; out->S_time = 1; }
  }
  // Stage 1b: per-axis chirp-z (Ma -> Ba).
  out->P_space_x = std::max(kMinFFT, pow2_at_least((int64_t)g->mx + g->bx - 1));
  out->P_space_y = g->kind == FBST_URA ? std::max(kMinFFT, pow2_at_least((int64_t)g->my + g->by - 1)) : 0;
  // Stage 2.
  out->P_gs = std::max(kMinFFT, pow2_at_least(2 * (int64_t)L - 1));
  {
    const int P1 = std::max(kMinFFT, pow2_at_least((int64_t)L + N - 1));
    const int P2 = std::max(kMinFFT, pow2_at_least((int64_t)L / 2 + N - 1));
    const bool ok1 = P1 == out->P_gs || 2 * P1 == out->P_gs;
    const bool ok2 = P2 == out->P_gs || 2 * P2 == out->P_gs;
    const double c1 = 2.0 * P1 * ilog2(P1), c2 = 3.0 * P2 * ilog2(P2);
    if (ok2 && (!ok1 || c2 < c1)) { out->P_rec = P2; out->S_rec = 2; }
    else if (ok1) { out->P_rec = P1; out->S_rec = 1; }
    else return FBST_ERR_UNSUPPORTED;
  }
  if (out->P_time > kMaxFFT || out->P_space_x > kMaxFFT || out->P_space_y > kMaxFFT ||
      out->P_gs > kMaxFFT || out->P_rec > kMaxFFT)
    return FBST_ERR_UNSUPPORTED;
  if (M > kMaxFFT || B > 65535) return FBST_ERR_UNSUPPORTED;

  out->stage2 = band->stage2 == FBST_STAGE2_AUTO ? FBST_STAGE2_GS_IR1 : band->stage2;

  // Eq. (8): the largest spread of element delays over the (physical) beams, in samples;
  // Eq. (4): epsilon * T_theta / (N T_s) with T_theta = spread + (N-1) T_s.
  double spread = 0.0;
  for (int a = 0; a < g->bx; ++a) {
    for (int c = 0; c < g->by; ++c) {
      const double u = -1.0 + 2.0 * a / g->bx;
      const double v = g->kind == FBST_URA ? -1.0 + 2.0 * c / g->by : 0.0;
      if (u * u + v * v > 1.0 + 1e-12) continue;
      spread = std::max(spread, out->rho * (std::fabs(u) * (g->mx - 1) + std::fabs(v) * (g->my - 1)));
    }
  }
  const double eps = (double)out->eps_num / (double)out->eps_den;
  out->snapshot_bound = spread;
  out->gamma_bound = eps * (spread + (N - 1)) / N;
  out->warn_snapshots = N <= spread;
  out->warn_gamma = (double)L / N <= out->gamma_bound;

  // Memory accounting.
  const size_t c64 = sizeof(float2);
  size_t tb = kTwiddleSize * (sizeof(float2) + sizeof(double2));
  tb += c64 * ((size_t)N + (size_t)out->S_time * out->P_time + L);
  tb += c64 * (size_t)L * (g->mx + out->P_space_x + g->bx);
  if (g->kind == FBST_URA && !(g->mx == g->my && g->bx == g->by))
    tb += c64 * (size_t)L * (g->my + out->P_space_y + g->by);
  tb += sizeof(double2) * (size_t)B * L;
  if (out->stage2 == FBST_STAGE2_GS || out->stage2 == FBST_STAGE2_GS_IR1) {
    tb += c64 * (size_t)B * (out->stage2 == FBST_STAGE2_GS_IR1 ? 3 : 2) * out->P_gs;
    tb += c64 * ((size_t)L + (size_t)out->S_rec * out->P_rec + N);
  } else {
    // G_b in complex64 (FP32 apply), or its tensor-core planes (8 bytes per entry in every
    // variant; the complex64 G_b is freed once they are built).
    tb += c64 * (size_t)B * N * L;
    if (out->stage2 == FBST_STAGE2_DENSE_F16X3) tb += sizeof(int) * (size_t)B;  // beam scales of G
  }
  out->table_bytes = tb;
  out->workspace_bytes = c64 * (size_t)band->max_blocks * ((size_t)L * M + (size_t)B * L);
  // The pre-split right-hand sides of the BF16x3 and TF32 tensor-core variants.
  if (out->stage2 == FBST_STAGE2_DENSE_BF16X3 || out->stage2 == FBST_STAGE2_DENSE_TF32)
    out->workspace_bytes += c64 * (size_t)B * (((size_t)band->max_blocks + 15) / 16 * 16) * L;
  // The block maxima of w behind the block scales of the FP16-split variant.
  if (out->stage2 == FBST_STAGE2_DENSE_F16X3) out->workspace_bytes += sizeof(unsigned) * (size_t)band->max_blocks;
  return FBST_OK;
}

namespace fbst {

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------
struct rat_consts {
  int64_t en, ed;  // epsilon = en/ed
  int64_t fp, fq;  // fb = fp/fq, rho = fp/(2 fq + fp)
  int N, L;
};

// exp(i*pi*q/D) with q reduced exactly modulo 2D before the FP64 sincospi.
__device__ __forceinline__ double2 expi_pi(int64_t q, int64_t D) {
  const int64_t twoD = 2 * D;
  int64_t m = q % twoD;
  if (m < 0) m += twoD;
  if (m >= D) m -= twoD;  // now -D <= m < D
  double s, c;
  sincospi((double)m / (double)D, &s, &c);
  return make_double2(c, s);
}

// sin(pi*q/D) with the same exact reduction.
__device__ __forceinline__ double sinpi_rat(int64_t q, int64_t D) {
  const int64_t twoD = 2 * D;
  int64_t m = q % twoD;
  if (m < 0) m += twoD;
  if (m >= D) m -= twoD;
  return sinpi((double)m / (double)D);
}

// sum_{m=0}^{count-1} exp(i*sign*theta*m) with theta = pi*Y/D (closed-form Dirichlet kernel):
// exp(i*sign*theta*(count-1)/2) * sin(count*theta/2) / sin(theta/2), or count if theta = 0 mod 2pi.
__device__ double2 dirichlet_sum(int64_t Y, int64_t D, int count, int sign) {
  int64_t r = Y % (2 * D);
  if (r < 0) r += 2 * D;
  if (r == 0) return make_double2((double)count, 0.0);
  const double num = sinpi_rat((int64_t)count * Y, 2 * D);
  const double den = sinpi_rat(Y, 2 * D);
  const double2 ph = expi_pi((int64_t)sign * (int64_t)(count - 1) * Y, 2 * D);
  const double q = num / den;
  return make_double2(ph.x * q, ph.y * q);
}

// Position of circular index k (0 <= k < P) in a kernel supported on d in [dmin, dmax],
// dmin <= 0 <= dmax, dmax - dmin < P; returns false outside the support.
__device__ __forceinline__ bool circ_index(int k, int P, int dmin, int dmax, int* d) {
  if (k <= dmax) { *d = k; return true; }
  if (k - P >= dmin) { *d = k - P; return true; }
  return false;
}

// Twiddle ladder: for every power of two M = 2..kTwiddleSize, exp(-2*pi*i*k/M) for k < M/2 at
// index M/2 - 1 + k (4095 entries; the last slot holds 1). A pass of radix R over sub-transforms
// of size NS needs exp(-2*pi*i*s*k/(NS*R)) = the ladder entry k of M = NS*R/s for k < NS, so the
// threads of a warp (consecutive k) read consecutive entries.
__global__ void k_twiddles(double2* tw64, float2* tw32) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < kTwiddleSize; idx += gridDim.x * blockDim.x) {
    double2 w = make_double2(1.0, 0.0);
    if (idx < kTwiddleSize - 1) {
      int half = 1;  // M / 2: the largest power of two <= idx + 1
      while (2 * half <= idx + 1) half *= 2;
      const int k = idx - (half - 1);
      w = expi_pi(-2 * (int64_t)k, 2 * half);  // exp(-2*pi*i*k/M), M = 2*half
    }
    tw64[idx] = w;
    tw32[idx] = make_float2((float)w.x, (float)w.y);
  }
}

// Stage 1a (Sec. IV, first sum): yhat[k] = sum_n y[n] exp(-2*pi*i*eps*(k + 1 - L/2)*n/L).
// Output k = h*Lh + i (Lh = L/S) uses c_h = h*Lh + 1 - L/2 and, with i*n = (i^2 + n^2 - (i-n)^2)/2,
//   pre[n]    = exp(-i*pi*eps*n^2/L)
//   g_h(d)    = exp(+i*pi*eps*(d^2 + 2 c_h d)/L),      d = i - n in [-(N-1), Lh-1]
//   post[k]   = exp(-i*pi*eps*(i^2 + 2 c_h i)/L).
__global__ void k_time_tables(float2* pre, float2* post, rat_consts rc, int S) {
  const int N = rc.N, L = rc.L, Lh = L / S;
  const int64_t D = rc.ed * L;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N + L; k += gridDim.x * blockDim.x) {
    if (k < N) {
      const double2 v = expi_pi(-rc.en * (int64_t)k * k, D);
      pre[k] = make_float2((float)v.x, (float)v.y);
    } else {
      const int kk = k - N, h = kk / Lh, i = kk % Lh;
      const int64_t ch = (int64_t)h * Lh + 1 - L / 2;
      const double2 v = expi_pi(-rc.en * ((int64_t)i * i + 2 * ch * i), D);
      post[kk] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__global__ void k_time_kernel_rows(double2* rows, rat_consts rc, int S, int P) {
  const int N = rc.N, L = rc.L, Lh = L / S;
  const int64_t D = rc.ed * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S * P; idx += gridDim.x * blockDim.x) {
    const int h = idx / P, k = idx % P;
    const int64_t ch = (int64_t)h * Lh + 1 - L / 2;
    int d;
    double2 v = make_double2(0.0, 0.0);
    if (circ_index(k, P, -(N - 1), Lh - 1, &d)) v = expi_pi(rc.en * ((int64_t)d * d + 2 * ch * d), D);
    rows[idx] = v;
  }
}

// Stage 1b (Sec. IV second sum, App. B per axis): for frequency ell, kappa = rho*(1/fb + eps*ell'/L)
// = Kn/Kd with Kn = fq*ed*L + fp*en*ell', Kd = (2 fq + fp)*ed*L. The steering
// exp(2*pi*i*kappa*u_b*m) with u_b = (2b - Ba)/Ba is a chirp-z: with 2bm = b^2 + m^2 - (b-m)^2,
//   pre[m]  = exp(2*pi*i*kappa*(m^2 - Ba*m)/Ba), kernel(d) = exp(-2*pi*i*kappa*d^2/Ba),
//   post[b] = exp(2*pi*i*kappa*b^2/Ba),          d = b - m in [-(Ma-1), Ba-1].
__device__ __forceinline__ int64_t kappa_num(const rat_consts& rc, int ell) {
  const int64_t lp = (int64_t)ell + 1 - rc.L / 2;
  return rc.fq * rc.ed * rc.L + rc.fp * rc.en * lp;
}
__device__ __forceinline__ int64_t kappa_den(const rat_consts& rc) { return (2 * rc.fq + rc.fp) * rc.ed * rc.L; }

__global__ void k_space_tables(float2* pre, float2* post, rat_consts rc, int Ma, int Ba) {
  const int ell = blockIdx.y;
  const int64_t Kn = kappa_num(rc, ell), D = kappa_den(rc) * Ba;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Ma + Ba; k += gridDim.x * blockDim.x) {
    if (k < Ma) {
      const double2 v = expi_pi(2 * Kn * ((int64_t)k * k - (int64_t)Ba * k), D);
      pre[(size_t)ell * Ma + k] = make_float2((float)v.x, (float)v.y);
    } else {
      const int b = k - Ma;
      const double2 v = expi_pi(2 * Kn * ((int64_t)b * b), D);
      post[(size_t)ell * Ba + b] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__global__ void k_space_kernel_rows(double2* rows, rat_consts rc, int Ma, int Ba, int P) {
  const int ell = blockIdx.y;
  const int64_t Kn = kappa_num(rc, ell), D = kappa_den(rc) * Ba;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    int d;
    double2 v = make_double2(0.0, 0.0);
    if (circ_index(k, P, -(Ma - 1), Ba - 1, &d)) v = expi_pi(-2 * Kn * ((int64_t)d * d), D);
    rows[(size_t)ell * P + k] = v;
  }
}

// Reconstruction F_u (Eq. (7)) as a chirp-z in n (Sec. V): bhat[n] = sum_ell beta[ell]
// exp(2*pi*i*eps*ell'*n/L). Input ell = h*Lr + i uses c_h = h*Lr + 1 - L/2 and, with
// i*n = (i^2 + n^2 - (n-i)^2)/2,
//   pre_h[i] = exp(i*pi*eps*(i^2 + 2 c_h i)/L), q_h(d) = exp(-i*pi*eps*(d^2 - 2 c_h d)/L),
//   post[n]  = exp(i*pi*eps*n^2/L),                d = n - i in [-(Lr-1), N-1].
__global__ void k_rec_tables(float2* pre, float2* post, rat_consts rc, int S) {
  const int N = rc.N, L = rc.L, Lr = L / S;
  const int64_t D = rc.ed * L;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L + N; k += gridDim.x * blockDim.x) {
    if (k < L) {
      const int h = k / Lr, i = k % Lr;
      const int64_t ch = (int64_t)h * Lr + 1 - L / 2;
      const double2 v = expi_pi(rc.en * ((int64_t)i * i + 2 * ch * i), D);
      pre[k] = make_float2((float)v.x, (float)v.y);
    } else {
      const int n = k - L;
      const double2 v = expi_pi(rc.en * (int64_t)n * n, D);
      post[n] = make_float2((float)v.x, (float)v.y);
    }
  }
}

__global__ void k_rec_kernel_rows(double2* rows, rat_consts rc, int S, int P) {
  const int N = rc.N, L = rc.L, Lr = L / S;
  const int64_t D = rc.ed * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S * P; idx += gridDim.x * blockDim.x) {
    const int h = idx / P, k = idx % P;
    const int64_t ch = (int64_t)h * Lr + 1 - L / 2;
    int d;
    double2 v = make_double2(0.0, 0.0);
    if (circ_index(k, P, -(Lr - 1), N - 1, &d)) v = expi_pi(-rc.en * ((int64_t)d * d - 2 * ch * d), D);
    rows[idx] = v;
  }
}

// In-place FP64 FFT of `rows` contiguous rows of length P (one CTA per row).
template <int P>
__global__ void k_fft64_rows(double2* data, const double2* __restrict__ tw, int dir) {
  constexpr int E = P >= 2048 ? 16 : (P >= 8 ? 8 : 2);
  constexpr int T = P / E;
  extern __shared__ double2 sm64[];
  double2* row = data + (size_t)blockIdx.x * P;
  const int t = threadIdx.x;
  double2 v[1][E];
#pragma unroll
  for (int r = 0; r < E; ++r) v[0][r] = row[t + T * r];
  if (dir < 0) block_fft<P, E, 1, -1>(v, sm64, tw, t);
  else block_fft<P, E, 1, +1>(v, sm64, tw, t);
#pragma unroll
  for (int r = 0; r < E; ++r) row[t + T * r] = v[0][r];
}

__global__ void k_to_c64(const double2* __restrict__ src, float2* __restrict__ dst, size_t n, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = src[i];
    dst[i] = make_float2((float)(v.x * scale), (float)(v.y * scale));
  }
}

__global__ void k_scale64(double2* data, size_t n, double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    data[i].x *= scale;
    data[i].y *= scale;
  }
}

// Toeplitz generator of A_b (Sec. V): [A_b]_{ell,k} = a_b(k - ell) with
//   a_b(d) = sum_{m,n} exp(i*(omega_k - omega_ell)*(t_n - tau_m)) + delta*[d == 0]
//          = D_N(2*pi*eps*d/L) * sum_m exp(-2*pi*i*eps*rho*d*(u_b.p_m)/L) + delta*[d == 0],
// D_N(x) = sum_{n<N} exp(i*x*n). The element sum factors over the two axes of a rectangular array.
// Each angle is pi * (integer)/(integer), so the closed forms use exact reductions.
__global__ void k_generators(double2* gen, rat_consts rc, int bx, int by, int mx, int my, double delta) {
  const int b = blockIdx.y;
  const int ia = b / by, ic = b % by;
  const int L = rc.L;
  const int64_t rden = 2 * rc.fq + rc.fp;  // rho = fp / rden
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < L; d += gridDim.x * blockDim.x) {
    // time factor: theta = 2*pi*eps*d/L = pi * (2 en d) / (ed L)
    const double2 dn = dirichlet_sum(2 * rc.en * d, rc.ed * L, rc.N, +1);
    // x axis: theta = 2*pi*eps*rho*d*u_a/L, u_a = (2a - bx)/bx -> pi * Y / D
    const double2 ax = dirichlet_sum(2 * rc.en * rc.fp * (int64_t)d * (2 * ia - bx),
                                     rc.ed * rden * L * (int64_t)bx, mx, -1);
    double2 af = ax;
    if (my > 1 || by > 1) {
      const double2 ay = dirichlet_sum(2 * rc.en * rc.fp * (int64_t)d * (2 * ic - by),
                                       rc.ed * rden * L * (int64_t)by, my, -1);
      af = cmul(ax, ay);
    }
    double2 a = cmul(dn, af);
    if (d == 0) a.x += delta;
    gen[(size_t)b * L + d] = a;
  }
}

// sum_{m<count} exp(-2*pi*i*phi*m) for a real phi (cycles) in FP64: exp(-i*pi*phi*(count-1)) *
// sin(pi*count*phi) / sin(pi*phi), or count when phi is an integer.
__device__ double2 dirichlet_real(double phi, int count) {
  const double den = sinpi(phi);
  if (den == 0.0) return make_double2((double)count, 0.0);   // every term is 1
  double s, c;
  sincospi(-phi * (count - 1), &s, &c);
  const double q = sinpi(phi * count) / den;
  return make_double2(c * q, s * q);
}

// Toeplitz generator of the A of an arbitrary direction (u, v) (Sec. VIII-A: an off-grid beam has
// its own regularised least-squares problem): as k_generators, with the element sums evaluated in
// FP64 from the direction cosines (no exact reduction: the phases eps*rho*d*u/L are below 2 cycles,
// and their FP64 rounding is far below the FP32 results built from them). dirs: [count][2].
__global__ void k_generators_dir(double2* gen, rat_consts rc, const double* __restrict__ dirs, int mx, int my,
                                 double delta) {
  const int k = blockIdx.y;
  const int L = rc.L;
  const double eps = (double)rc.en / (double)rc.ed;
  const double rho = (double)rc.fp / (double)(2 * rc.fq + rc.fp);
  const double u = dirs[2 * k], v = dirs[2 * k + 1];
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < L; d += gridDim.x * blockDim.x) {
    const double2 dn = dirichlet_sum(2 * rc.en * d, rc.ed * L, rc.N, +1);
    double2 af = dirichlet_real(eps * rho * d * u / L, mx);
    if (my > 1) af = cmul(af, dirichlet_real(eps * rho * d * v / L, my));
    double2 a = cmul(dn, af);
    if (d == 0) a.x += delta;
    gen[(size_t)k * L + d] = a;
  }
}

// Toeplitz generator of A_b for a linear array at arbitrary positions p_m (Sec. IX: only the element
// sum changes off the grid): a_b(d) = D_N(2*pi*eps*d/L) * sum_m exp(-2*pi*i*eps*rho*u_b*p_m*d/L)
// + delta*[d == 0]. One CTA per beam; warp w owns the d range [w*L/8, (w+1)*L/8) and sums over
// the elements 32 at a time, lane l taking element m: z_m = exp(-2*pi*i*alpha*p_m) with
// alpha = eps*rho*u_b/L, z_m^d by repeated products from z_m^{d0} (FP64 sincospi once per element
// and warp; the products lose about d ulps), then a warp reduction per d.
__global__ void __launch_bounds__(256) k_generators_positions(double2* gen, rat_consts rc, const double* __restrict__ pos,
                                                              const double* __restrict__ pos_y, int M, int bx, int by,
                                                              double delta) {
  extern __shared__ double2 accg[];  // [L]
  const int b = blockIdx.x, L = rc.L;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double eps = (double)rc.en / (double)rc.ed;
  const double rho = (double)rc.fp / (double)(2 * rc.fq + rc.fp);
  // Beam b = bu * by + bv at (u, v) = (-1 + 2 bu / bx, -1 + 2 bv / by); the element's delay per unit
  // d is alpha_x x_m + alpha_y y_m (y = 0 for a linear array, pos_y = NULL).
  const double ax = eps * rho * (-1.0 + 2.0 * (b / by) / bx) / L;
  const double ay = pos_y ? eps * rho * (-1.0 + 2.0 * (b % by) / by) / L : 0.0;
  const int d0 = (int)((long long)L * warp / 8), d1 = (int)((long long)L * (warp + 1) / 8);
  for (int d = d0 + lane; d < d1; d += 32) accg[d] = make_double2(0.0, 0.0);
  __syncwarp();
  for (int m0 = 0; m0 < M; m0 += 32) {
    const int m = m0 + lane;
    double2 z = make_double2(1.0, 0.0), zp = make_double2(0.0, 0.0);
    if (m < M) {
      const double dly = ax * pos[m] + (pos_y ? ay * pos_y[m] : 0.0);
      double sn, cs;
      sincospi(-2.0 * dly, &sn, &cs);
      z = make_double2(cs, sn);
      sincospi(-2.0 * dly * d0, &sn, &cs);
      zp = make_double2(cs, sn);                // z^{d0}
    }
    for (int d = d0; d < d1; ++d) {
      double2 v = zp;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      }
      if (lane == 0) accg[d] = cadd(accg[d], v);
      zp = cmul(zp, z);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < L; d += blockDim.x) {
    double2 a = cmul(dirichlet_sum(2 * rc.en * d, rc.ed * L, rc.N, +1), accg[d]);
    if (d == 0) a.x += delta;
    gen[(size_t)b * L + d] = a;
  }
}

// Type-1 NUFFT tables of the non-uniform stage 1b (Sec. IX, Eq. (16)). With u_b = 2(b - B/2)/B the
// element sum is w_b[ell] = sum_m yhat[m, ell] exp(2*pi*i*(b - B/2)*x_m), x_m = 2*kappa_ell*p_m/B
// (cycles; kappa_ell = rho*(1/fb + eps*ell'/L)): a type-1 transform of the strengths yhat[., ell] at
// the points x_m onto the centred modes b - B/2. Each point spreads onto the W grid points
// j0, ..., j0 + W - 1 (mod nf) of the nf-point grid around its grid coordinate g = nf*x_m with the
// "exponential of semicircle" kernel phi(z) = exp(beta*(sqrt(1 - z^2) - 1)), z = (j - g)/(W/2). The
// table keeps j0 and g - j0 per (ell, m), computed in FP64 (g - j0 lies in (W/2 - 1, W/2], so its
// float keeps about 5e-7 absolute); the run-time kernel evaluates the W weights from it.
__global__ void k_nufft_tables(int* __restrict__ j0, float* __restrict__ dg, rat_consts rc, const double* __restrict__ pos,
                               int M, int B, int nf, int W) {
  const int L = rc.L;
  const double eps = (double)rc.en / (double)rc.ed;
  const double fbv = (double)rc.fp / (double)rc.fq;
  const double rho = (double)rc.fp / (double)(2 * rc.fq + rc.fp);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)L * M; i += (long long)gridDim.x * blockDim.x) {
    const int ell = (int)(i / M), m = (int)(i % M);
    const double kappa = rho * (1.0 / fbv + eps * (double)(ell + 1 - L / 2) / L);
    double g = nf * (2.0 * kappa * pos[m] / B);          // grid coordinate of x_m
    g -= nf * floor(g / nf);                              // into [0, nf)
    const double first = ceil(g - 0.5 * W);
    dg[i] = (float)(g - first);
    int jj = (int)first % nf;
    if (jj < 0) jj += nf;
    j0[i] = jj;
  }
}

// FP64 Levinson recursion for x = A^{-1} e_0, A Hermitian positive definite Toeplitz with first
// column c[d] = conj(a(d)). Keeps f_k solving A_k f_k = e_0; with eps_k = sum_{i<k} c[k-i] f_k[i]
// the extension is f_{k+1}[i] = (f_k[i] - eps_k conj(f_k[k-i])) / (1 - |eps_k|^2) (f_k[k] = 0).
// One CTA per beam; writes FBST_ERR_NUMERIC to *status if a pivot is not positive.
__global__ void k_levinson(const double2* __restrict__ gen, double2* __restrict__ xout, int L, int* status) {
  extern __shared__ double2 smL[];
  double2* f = smL;
  double2* c = smL + L;
  double2* red = smL + 2 * L;  // one partial per warp
  const int b = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  const int nwarp = (nth + 31) / 32;
  for (int i = tid; i < L; i += nth) {
    const double2 a = gen[(size_t)b * L + i];
    c[i] = make_double2(a.x, -a.y);
    f[i] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (tid == 0) f[0] = make_double2(1.0 / c[0].x, 0.0);
  __syncthreads();
  bool bad = !(c[0].x > 0.0);
  for (int k = 1; k < L && !bad; ++k) {
    double2 part = make_double2(0.0, 0.0);
    for (int i = tid; i < k; i += nth) part = cadd(part, cmul(c[k - i], f[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
      part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    double2 ef = make_double2(0.0, 0.0);
    for (int w = 0; w < nwarp; ++w) ef = cadd(ef, red[w]);
    const double den = 1.0 - (ef.x * ef.x + ef.y * ef.y);
    if (!(den > 1e-300)) {
      bad = true;  // identical in every thread (same ef)
    } else {
      const double inv = 1.0 / den;
      for (int i = tid; 2 * i <= k; i += nth) {
        const int j = k - i;
        const double2 fi = f[i], fj = f[j];
        const double2 ni = cscale(csub(fi, cmul(ef, cconj(fj))), inv);
        const double2 nj = cscale(csub(fj, cmul(ef, cconj(fi))), inv);
        f[i] = ni;
        if (j != i) f[j] = nj;
      }
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(status, (int)FBST_ERR_NUMERIC);
    return;
  }
  for (int i = tid; i < L; i += nth) xout[(size_t)b * L + i] = f[i];
}

int launch_levinson(const double2* gen, double2* x, int count, int L, int* status, cudaStream_t s) {
  const size_t lev_smem = (2 * (size_t)L + 32) * sizeof(double2);
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_levinson, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lev_smem));
  k_levinson<<<count, 256, lev_smem, s>>>(gen, x, L, status);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

// Rows for the Gohberg-Semencul spectra: row 2b = x_b / sqrt(x_0), row 2b+1 = Z J conj(x_b) / sqrt(x_0),
// both zero-padded to P.
__global__ void k_gs_rows(const double2* __restrict__ x, double2* __restrict__ rows, int L, int P, int* status) {
  const int b = blockIdx.y;
  const double x0 = x[(size_t)b * L].x;
  if (!(x0 > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(status, (int)FBST_ERR_NUMERIC);
    return;
  }
  const double s = rsqrt(x0);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    const double2 xr = k < L ? cscale(x[(size_t)b * L + k], s) : make_double2(0.0, 0.0);
    const double2 vr = (k >= 1 && k < L) ? cscale(cconj(x[(size_t)b * L + L - k]), s) : make_double2(0.0, 0.0);
    rows[((size_t)b * 2 + 0) * P + k] = xr;
    rows[((size_t)b * 2 + 1) * P + k] = vr;
  }
}

// Circulant embedding of A_b for the refinement residual: first column c with c[j] = A[j,0] =
// conj(a(j)) for j < L and c[P-j] = A[0,j] = a(j) for 0 < j < L, so (C beta)[i] = (A beta)[i] for
// i < L when beta is zero beyond L and P >= 2L-1.
__global__ void k_toeplitz_rows(const double2* __restrict__ gen, double2* __restrict__ rows, int L, int P) {
  const int b = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P; k += gridDim.x * blockDim.x) {
    double2 v = make_double2(0.0, 0.0);
    if (k < L) v = cconj(gen[(size_t)b * L + k]);
    else if (P - k < L) v = gen[(size_t)b * L + (P - k)];
    rows[(size_t)b * P + k] = v;
  }
}

// Dense operator G_b = F_u A_b^{-1} in FP64 (Sec. III-B): row n is conj(A_b^{-1} conj(f_n)) with
// f_n[ell] = exp(2*pi*i*eps*ell'*n/L), since A_b^{-T} = conj(A_b^{-1}). One CTA per (n, b).
template <int P>
__global__ void k_dense_G(const double2* __restrict__ XV64, float2* __restrict__ G, rat_consts rc,
                          const double2* __restrict__ tw) {
  constexpr int E = P >= 2048 ? 16 : (P >= 8 ? 8 : 2);
  constexpr int T = P / E;
  extern __shared__ double2 smG[];
  const int n = blockIdx.x, b = blockIdx.y, t = threadIdx.x, L = rc.L;
  const double2* Xb = XV64 + (size_t)b * 2 * P;
  double2 v[E], X[E], Vv[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    v[r] = i < L ? expi_pi(-2 * rc.en * ((int64_t)i + 1 - L / 2) * n, rc.ed * L) : make_double2(0.0, 0.0);
    X[r] = Xb[i];
    Vv[r] = Xb[P + i];
  }
  gs_apply<P, E>(v, X, Vv, smG, tw, t, L);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    if (i < L) G[((size_t)b * rc.N + n) * L + i] = make_float2((float)v[r].x, (float)-v[r].y);
  }
}

// ---------------------------------------------------------------------------------------------
// Host-side launch helpers
// ---------------------------------------------------------------------------------------------
template <int P>
static int fft64_rows_P(double2* data, int rows, const double2* tw, int dir, cudaStream_t s) {
  constexpr int E = P >= 2048 ? 16 : (P >= 8 ? 8 : 2);
  const size_t smem = sizeof(double2) * fft_smem_elems<double2>(P);
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_fft64_rows<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (rows > 0) k_fft64_rows<P><<<rows, P / E, smem, s>>>(data, tw, dir);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int fft64_rows(double2* data, int rows, int P, const double2* tw, int dir, cudaStream_t s) {
  switch (P) {
    case 16: return fft64_rows_P<16>(data, rows, tw, dir, s);
    case 32: return fft64_rows_P<32>(data, rows, tw, dir, s);
    case 64: return fft64_rows_P<64>(data, rows, tw, dir, s);
    case 128: return fft64_rows_P<128>(data, rows, tw, dir, s);
    case 256: return fft64_rows_P<256>(data, rows, tw, dir, s);
    case 512: return fft64_rows_P<512>(data, rows, tw, dir, s);
    case 1024: return fft64_rows_P<1024>(data, rows, tw, dir, s);
    case 2048: return fft64_rows_P<2048>(data, rows, tw, dir, s);
    case 4096: return fft64_rows_P<4096>(data, rows, tw, dir, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

template <int P>
static int dense_G_P(const double2* XV64, float2* G, rat_consts rc, int B, const double2* tw, cudaStream_t s) {
  constexpr int E = P >= 2048 ? 16 : (P >= 8 ? 8 : 2);
  const size_t smem = 2 * sizeof(double2) * fft_smem_elems<double2>(P);
  FBST_CUDA_TRY(cudaFuncSetAttribute(k_dense_G<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_dense_G<P><<<dim3(rc.N, B), P / E, smem, s>>>(XV64, G, rc, tw);
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

static int dense_G(const double2* XV64, float2* G, rat_consts rc, int B, int P, const double2* tw, cudaStream_t s) {
  switch (P) {
    case 16: return dense_G_P<16>(XV64, G, rc, B, tw, s);
    case 32: return dense_G_P<32>(XV64, G, rc, B, tw, s);
    case 64: return dense_G_P<64>(XV64, G, rc, B, tw, s);
    case 128: return dense_G_P<128>(XV64, G, rc, B, tw, s);
    case 256: return dense_G_P<256>(XV64, G, rc, B, tw, s);
    case 512: return dense_G_P<512>(XV64, G, rc, B, tw, s);
    case 1024: return dense_G_P<1024>(XV64, G, rc, B, tw, s);
    case 2048: return dense_G_P<2048>(XV64, G, rc, B, tw, s);
    case 4096: return dense_G_P<4096>(XV64, G, rc, B, tw, s);
    default: return FBST_ERR_UNSUPPORTED;
  }
}

static int grid_for(size_t n, int threads) {
  size_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

#define FBST_TRY(expr)          \
  do {                          \
    const int fbst_r_ = (expr); \
    if (fbst_r_ != FBST_OK) return fbst_r_; \
  } while (0)

// Shape parameter of the spreading kernel for a width of W grid points on a 2x oversampled grid
// (the choice of Barnett, Magland and af Klinteberg for the "exponential of semicircle" kernel).
double nufft_beta(int W) { return 2.30 * W; }

// Gauss-Legendre nodes and weights on [-1, 1] (n points, FP64): Newton on P_n from the classic
// cosine initial guess, P_n and P_n' by the three-term recurrence.
static void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Deconvolution factors of the non-uniform stage 1b: spreading with psi(s) = phi(2s/W) and an
// unnormalised inverse-sign FFT of the grid give, at mode k, sum_m c_m exp(2*pi*i*k*x_m) times
// Psi(k/nf) = integral psi(s) exp(2*pi*i*(k/nf)*s) ds = W * integral_0^1 phi(z) cos(pi*(k/nf)*W*z) dz
// (phi even), up to the aliasing error the kernel width sets. Beam b reads mode k = b - B/2; its
// factor 1/Psi is computed here by 200-point Gauss-Legendre quadrature in FP64 and rounded once.
// 1 / (W * kernel Fourier transform) at the modes b - B/2 of an axis of B beams on an nf-point grid.
static int nufft_deconv_axis(const fbst_plan_s* p, int B, int nf, float* dst, cudaStream_t s) {
  const int W = p->nu_w;
  const double beta = nufft_beta(W);
  constexpr int kQ = 200;
  double xq[kQ], wq[kQ];
  gauss_legendre(kQ, xq, wq);
  float* host = static_cast<float*>(std::malloc(sizeof(float) * B));
  if (!host) return FBST_ERR_OOM;
  for (int b = 0; b < B; ++b) {
    const double nu = (double)(b - B / 2) / nf;
    double acc = 0.0;
    for (int i = 0; i < kQ; ++i) {
      const double z = 0.5 * (xq[i] + 1.0);              // [0, 1]
      acc += 0.5 * wq[i] * std::exp(beta * (std::sqrt(std::max(0.0, 1.0 - z * z)) - 1.0)) * std::cos(M_PI * nu * W * z);
    }
    host[b] = (float)(1.0 / (W * acc));
  }
  const cudaError_t e = cudaMemcpyAsync(dst, host, sizeof(float) * B, cudaMemcpyHostToDevice, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  std::free(host);
  FBST_CUDA_TRY(e);
  FBST_CUDA_TRY(e2);
  return FBST_OK;
}

int nufft_deconv(fbst_plan_s* p, cudaStream_t s) {
  if (!p->nu_nfy) return nufft_deconv_axis(p, p->info.B, p->nu_nf, p->nu_deconv, s);
  FBST_TRY(nufft_deconv_axis(p, p->geom.bx, p->nu_nf, p->nu_deconv, s));
  return nufft_deconv_axis(p, p->geom.by, p->nu_nfy, p->nu_deconv_y, s);
}

int plan_toeplitz_generators(fbst_plan_s* p, double2* gen, cudaStream_t s) {
  const fbst_info& in = p->info;
  const int L = in.L, B = in.B;
  rat_consts rc{in.eps_num, in.eps_den, in.fb_num, in.fb_den, in.N, L};
  if (p->nu_nf) {
    FBST_CUDA_TRY(cudaFuncSetAttribute(k_generators_positions, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(L * sizeof(double2))));
    k_generators_positions<<<B, 256, L * sizeof(double2), s>>>(gen, rc, p->pos, p->nu_nfy ? p->pos_y : nullptr, in.M,
                                                                p->geom.bx, p->geom.by, in.delta);
  } else {
    k_generators<<<dim3(grid_for(L, 256) > 64 ? 64 : grid_for(L, 256), B), 256, 0, s>>>(
        gen, rc, p->geom.bx, p->geom.by, p->geom.mx, p->geom.my, in.delta);
  }
  FBST_CUDA_TRY(cudaGetLastError());
  return FBST_OK;
}

int build_plan_tables(fbst_plan_s* p, cudaStream_t s) {
  const fbst_info& in = p->info;
  const int N = in.N, L = in.L, B = in.B;
  rat_consts rc{in.eps_num, in.eps_den, in.fb_num, in.fb_den, N, L};

  k_twiddles<<<16, 256, 0, s>>>(p->tw64, p->tw32);
  FBST_CUDA_TRY(cudaGetLastError());

  // Scratch for FP64 kernel rows: the largest user below.
  size_t scratch_elems = (size_t)in.S_time * in.P_time;
  scratch_elems = std::max(scratch_elems, (size_t)L * in.P_space_x);
  scratch_elems = std::max(scratch_elems, (size_t)L * in.P_space_y);
  scratch_elems = std::max(scratch_elems, (size_t)in.S_rec * in.P_rec);
  scratch_elems = std::max(scratch_elems, (size_t)B * 2 * in.P_gs);
  double2* scratch = nullptr;
  double2* gen = nullptr;
  FBST_TRY(plan_alloc_n(p, &scratch, scratch_elems));
  {
    const int r = plan_alloc_n(p, &gen, (size_t)B * L);
    if (r != FBST_OK) {
      plan_free(p, scratch);
      return r;
    }
  }
  int rc_status = FBST_OK;

  do {
    // Stage 1a tables.
    k_time_tables<<<grid_for(N + L, 256), 256, 0, s>>>(p->pre_t, p->post_t, rc, in.S_time);
    k_time_kernel_rows<<<grid_for((size_t)in.S_time * in.P_time, 256), 256, 0, s>>>(scratch, rc, in.S_time, in.P_time);
    if ((rc_status = fft64_rows(scratch, in.S_time, in.P_time, p->tw64, -1, s)) != FBST_OK) break;
    k_to_c64<<<grid_for((size_t)in.S_time * in.P_time, 256), 256, 0, s>>>(scratch, p->gspec_t, (size_t)in.S_time * in.P_time, 1.0 / in.P_time);

    // Stage 1b tables: the NUFFT tables of a non-uniform array, else one chirp-z set per axis.
    if (p->nu_nf) {
      // One table per axis: x against the bx beams along u, y against the by beams along v.
      k_nufft_tables<<<grid_for((size_t)L * in.M, 256), 256, 0, s>>>(p->nu_j0, p->nu_dg, rc, p->pos, in.M,
                                                                    p->geom.bx, p->nu_nf, p->nu_w);
      if (p->nu_nfy)
        k_nufft_tables<<<grid_for((size_t)L * in.M, 256), 256, 0, s>>>(p->nu_j0y, p->nu_dgy, rc, p->pos_y, in.M,
                                                                      p->geom.by, p->nu_nfy, p->nu_w);
      FBST_CUDA_TRY(cudaGetLastError());
      if ((rc_status = nufft_deconv(p, s)) != FBST_OK) break;
    }
    for (int a = 0; a < (p->nu_nf ? 0 : p->n_axes); ++a) {
      fbst_axis_tables& ax = p->ax[a];
      k_space_tables<<<dim3(grid_for(ax.Ma + ax.Ba, 256) > 64 ? 64 : grid_for(ax.Ma + ax.Ba, 256), L), 256, 0, s>>>(ax.pre, ax.post, rc, ax.Ma, ax.Ba);
      k_space_kernel_rows<<<dim3(grid_for(ax.P, 256) > 64 ? 64 : grid_for(ax.P, 256), L), 256, 0, s>>>(scratch, rc, ax.Ma, ax.Ba, ax.P);
      if ((rc_status = fft64_rows(scratch, L, ax.P, p->tw64, -1, s)) != FBST_OK) break;
      k_to_c64<<<grid_for((size_t)L * ax.P, 256), 256, 0, s>>>(scratch, ax.kspec, (size_t)L * ax.P, 1.0 / ax.P);
    }
    if (rc_status != FBST_OK) break;
    FBST_CUDA_TRY(cudaGetLastError());

    // Toeplitz generators (closed form on the grid, direct FP64 sums over a non-uniform array's
    // positions) and the solve for x_b (Levinson or superfast).
    if ((rc_status = plan_toeplitz_generators(p, gen, s)) != FBST_OK) break;
    if ((rc_status = solve_generators(p, gen, p->x64, B, p->band.generator_solver, s)) != FBST_OK) break;

    // Gohberg-Semencul spectra (FP64, kept in scratch for the dense build).
    const int Pg = in.P_gs;
    k_gs_rows<<<dim3(grid_for(Pg, 256) > 64 ? 64 : grid_for(Pg, 256), B), 256, 0, s>>>(p->x64, scratch, L, Pg, p->d_status);
    if ((rc_status = fft64_rows(scratch, 2 * B, Pg, p->tw64, -1, s)) != FBST_OK) break;
    k_scale64<<<grid_for((size_t)B * 2 * Pg, 256), 256, 0, s>>>(scratch, (size_t)B * 2 * Pg, 1.0 / Pg);
    FBST_CUDA_TRY(cudaGetLastError());

    if (in.stage2 == FBST_STAGE2_GS || in.stage2 == FBST_STAGE2_GS_IR1) {
      k_to_c64<<<grid_for((size_t)B * 2 * Pg, 256), 256, 0, s>>>(scratch, p->XV, (size_t)B * 2 * Pg, 1.0);
      if (in.stage2 == FBST_STAGE2_GS_IR1) {
        double2* arows = nullptr;
        if ((rc_status = plan_alloc_n(p, &arows, (size_t)B * Pg)) != FBST_OK) break;
        k_toeplitz_rows<<<dim3(grid_for(Pg, 256) > 64 ? 64 : grid_for(Pg, 256), B), 256, 0, s>>>(gen, arows, L, Pg);
        rc_status = fft64_rows(arows, B, Pg, p->tw64, -1, s);
        if (rc_status == FBST_OK)
          k_to_c64<<<grid_for((size_t)B * Pg, 256), 256, 0, s>>>(arows, p->Aspec, (size_t)B * Pg, 1.0 / Pg);
        plan_free(p, arows);
        if (rc_status != FBST_OK) break;
      }
      k_rec_tables<<<grid_for(L + N, 256), 256, 0, s>>>(p->pre_r, p->post_r, rc, in.S_rec);
      double2* qrows = nullptr;
      if ((rc_status = plan_alloc_n(p, &qrows, (size_t)in.S_rec * in.P_rec)) != FBST_OK) break;
      k_rec_kernel_rows<<<grid_for((size_t)in.S_rec * in.P_rec, 256), 256, 0, s>>>(qrows, rc, in.S_rec, in.P_rec);
      rc_status = fft64_rows(qrows, in.S_rec, in.P_rec, p->tw64, -1, s);
      if (rc_status == FBST_OK)
        k_to_c64<<<grid_for((size_t)in.S_rec * in.P_rec, 256), 256, 0, s>>>(qrows, p->qspec_r, (size_t)in.S_rec * in.P_rec, 1.0 / in.P_rec);
      plan_free(p, qrows);
      if (rc_status != FBST_OK) break;
    } else {
      if ((rc_status = dense_G(scratch, p->G, rc, B, Pg, p->tw64, s)) != FBST_OK) break;
      if (in.stage2 != FBST_STAGE2_DENSE_FP32) {
        if ((rc_status = build_dense_tc_operand(p, s)) != FBST_OK) break;
        plan_free(p, p->G);        // the tensor-core planes replace it (the free is stream-ordered)
        p->G = nullptr;
      }
    }
    FBST_CUDA_TRY(cudaGetLastError());
  } while (0);

  plan_free(p, scratch);
  plan_free(p, gen);
  FBST_CUDA_TRY(cudaStreamSynchronize(s));
  if (rc_status != FBST_OK) return rc_status;
  int st = 0;
  FBST_CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  return st;
}

int build_direction_x(fbst_plan_s* p, const double* dirs_dev, int count, double2* x, cudaStream_t s) {
  const fbst_info& in = p->info;
  const int L = in.L;
  rat_consts rc{in.eps_num, in.eps_den, in.fb_num, in.fb_den, in.N, L};
  double2* gen = nullptr;
  FBST_TRY(plan_alloc_n(p, &gen, (size_t)count * L));
  if (s != p->mem_stream && cudaStreamSynchronize(p->mem_stream) != cudaSuccess) {
    plan_free(p, gen);
    return FBST_ERR_CUDA;
  }
  const int gx = grid_for(L, 256) > 64 ? 64 : grid_for(L, 256);
  k_generators_dir<<<dim3(gx, count), 256, 0, s>>>(gen, rc, dirs_dev, p->geom.mx, p->geom.my, in.delta);
  const int r = solve_generators(p, gen, x, count, p->band.generator_solver, s);
  cudaStreamSynchronize(s);
  plan_free(p, gen);
  return r;
}

int build_direction_operators(fbst_plan_s* p, const double* dirs_dev, int count, float2* XV, float2* Aspec,
                              float2* pre_r, float2* qspec_r, float2* post_r, cudaStream_t s) {
  const fbst_info& in = p->info;
  const int N = in.N, L = in.L, Pg = in.P_gs;
  rat_consts rc{in.eps_num, in.eps_den, in.fb_num, in.fb_den, N, L};
  double2 *gen = nullptr, *x = nullptr, *rows = nullptr, *arows = nullptr, *qrows = nullptr;
  int r = FBST_OK;
  do {
    if ((r = plan_alloc_n(p, &gen, (size_t)count * L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &x, (size_t)count * L)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &rows, (size_t)count * 2 * Pg)) != FBST_OK) break;
    if (Aspec && (r = plan_alloc_n(p, &arows, (size_t)count * Pg)) != FBST_OK) break;
    if ((r = plan_alloc_n(p, &qrows, (size_t)in.S_rec * in.P_rec)) != FBST_OK) break;
    // Allocated in stream order on the plan's stream: make the blocks usable on `s`.
    if (s != p->mem_stream && cudaStreamSynchronize(p->mem_stream) != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    const int gx = grid_for(L, 256) > 64 ? 64 : grid_for(L, 256);
    k_generators_dir<<<dim3(gx, count), 256, 0, s>>>(gen, rc, dirs_dev, p->geom.mx, p->geom.my, in.delta);
    if ((r = solve_generators(p, gen, x, count, p->band.generator_solver, s)) != FBST_OK) break;
    k_gs_rows<<<dim3(grid_for(Pg, 256) > 64 ? 64 : grid_for(Pg, 256), count), 256, 0, s>>>(x, rows, L, Pg, p->d_status);
    if (cudaGetLastError() != cudaSuccess) { r = FBST_ERR_CUDA; break; }
    if ((r = fft64_rows(rows, 2 * count, Pg, p->tw64, -1, s)) != FBST_OK) break;
    k_to_c64<<<grid_for((size_t)count * 2 * Pg, 256), 256, 0, s>>>(rows, XV, (size_t)count * 2 * Pg, 1.0 / Pg);
    if (Aspec) {
      k_toeplitz_rows<<<dim3(grid_for(Pg, 256) > 64 ? 64 : grid_for(Pg, 256), count), 256, 0, s>>>(gen, arows, L, Pg);
      if ((r = fft64_rows(arows, count, Pg, p->tw64, -1, s)) != FBST_OK) break;
      k_to_c64<<<grid_for((size_t)count * Pg, 256), 256, 0, s>>>(arows, Aspec, (size_t)count * Pg, 1.0 / Pg);
    }
    k_rec_tables<<<grid_for(L + N, 256), 256, 0, s>>>(pre_r, post_r, rc, in.S_rec);
    k_rec_kernel_rows<<<grid_for((size_t)in.S_rec * in.P_rec, 256), 256, 0, s>>>(qrows, rc, in.S_rec, in.P_rec);
    if ((r = fft64_rows(qrows, in.S_rec, in.P_rec, p->tw64, -1, s)) != FBST_OK) break;
    k_to_c64<<<grid_for((size_t)in.S_rec * in.P_rec, 256), 256, 0, s>>>(qrows, qspec_r, (size_t)in.S_rec * in.P_rec,
                                                                       1.0 / in.P_rec);
    if (cudaGetLastError() != cudaSuccess) { r = FBST_ERR_CUDA; break; }
  } while (0);
  cudaStreamSynchronize(s);
  for (double2* q : {gen, x, rows, arows, qrows}) plan_free(p, q);
  if (r != FBST_OK) return r;
  int st = 0;
  FBST_CUDA_TRY(cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    cudaMemset(p->d_status, 0, sizeof(int));
    return st;
  }
  return FBST_OK;
}

}  // namespace fbst
