// Superfast solver for the stage-2 generators (Sec. V): x_b = A_b^{-1} e_0 for a Hermitian positive
// definite Toeplitz A_b, in O(L log^2 L) operations instead of the O(L^2) of the Levinson
// recursion, by the doubling (divide-and-conquer) form of the Schur algorithm.
//
// Notation. A has first column c (A[i][j] = c[i-j], c[-d] = conj(c[d])). The Levinson vectors f_k
// (A_k f_k = e_0, k x k leading block) and g_k = z f_k^#, f_k^#(z) = z^(k-1) conj(f_k(1/conj z)),
// obey [f_{k+1}, g_{k+1}] = [f_k, g_k] Lambda_k(z) with
//   Lambda_k(z) = 1/(1 - |eps_k|^2) [[1, -conj(eps_k) z], [-eps_k, z]],
// eps_k the coefficient k of c(z) f_k(z) (the residual of f_k one row beyond its block). The Schur
// residuals phi_k = c f_k and psi_k = c g_k (power series mod z^L) follow the same recursion, and
// eps_k = phi_k[k] / psi_k[k] (psi_k[k] = 1 in exact arithmetic), so the reflection coefficients
// come from the residuals alone, without the inner products of the Levinson recursion. Starting
// from f_1 = 1/c[0], g_1 = z/c[0], phi_1 = c/c[0], psi_1 = z c/c[0], the L - 1 steps k = 1..L-1
// give Theta(z) = Lambda_1 ... Lambda_{L-1} and x = f_L = (Theta_00 + z Theta_10)/c[0].
//
// Doubling. The eps_k of a step range [a, b) depend only on the coefficients [a, b) of phi_a and
// psi_a. A node [a, b) with midpoint m solves [a, m) (giving Theta_{a,m}), maps the windows to
// [phi_m, psi_m] = [phi_a, psi_a] Theta_{a,m} on the coefficients [m, b), solves [m, b) on them and
// returns Theta_{a,b} = Theta_{a,m} Theta_{m,b}. The window map and the product are polynomial
// products done by FP64 FFTs of size P = the power of two >= b - a: the wanted window
// coefficients lie above the wrap of the circular product, and the product's only wrapped
// coefficient (degree b - a of column 1, when P = b - a) lands on its constant term, which is zero
// because every Lambda's column 1 carries a factor z. Nodes of at most 32 steps run the steps
// themselves in one warp (lane j holds coefficient j; the shift by z is a shuffle). T(L) =
// 2 T(L/2) + O(L log L) = O(L log^2 L).
//
// One CTA per system, persistent over the systems; the recursion is an explicit stack walked by
// all threads alike; the windows and the per-depth results live in a global workspace slot of the
// CTA (L2-resident), the FFT exchange and spectra in shared memory. The window map of a node at
// depth l writes its right child's windows to a buffer of depth l + 1 (a left child reads a prefix
// of its parent's windows): in place it would overwrite coefficients that an ancestor's window map
// still reads.
#include "common.cuh"
#include "fft.cuh"
#include "launch_util.cuh"

namespace fbst {

namespace {

constexpr int kSfLeaf = 32;     // a node of at most this many steps runs them in one warp
constexpr int kSfThreads = 256;
constexpr int kSfMaxDepth = 12;  // depth of the recursion for L - 1 <= 32 * 2^12

// Coefficients of one result polynomial at depth l: a node there has at most
// ceil((L - 1) / 2^l) <= ((L - 1) >> l) + 1 steps and its polynomials one coefficient more.
__host__ __device__ inline int sf_slot_len(int L, int l) { return ((L - 1) >> l) + 2; }

// Depth of the deepest node: halve (rounding up) until a node fits a leaf.
__host__ __device__ inline int sf_depth(int L) {
  int d = 0;
  for (int s = L - 1; s > kSfLeaf; s = (s + 1) / 2) ++d;
  return d;
}

// Workspace of one CTA: per depth d a window buffer (phi then psi, win_len(d) coefficients each:
// the root's windows indexed by coefficient, deeper ones from the first coefficient of the right
// child that owns them), then per depth two result slots (left and right child) of four
// polynomials each.
__host__ __device__ inline int sf_win_len(int L, int d) { return d == 0 ? L : sf_slot_len(L, d); }

__host__ __device__ inline size_t sf_win_off(int L, int d) {
  size_t off = 0;
  for (int i = 0; i < d; ++i) off += 2 * (size_t)sf_win_len(L, i);
  return off;
}

__host__ __device__ inline size_t sf_ws_elems(int L) {
  const int d = sf_depth(L);
  size_t n = sf_win_off(L, d + 1);
  for (int l = 0; l <= d; ++l) n += 8 * (size_t)sf_slot_len(L, l);
  return n;
}

__device__ inline double2* sf_slot(double2* ws, int L, int l, int side) {
  size_t off = sf_win_off(L, sf_depth(L) + 1);
  for (int i = 0; i < l; ++i) off += 8 * (size_t)sf_slot_len(L, i);
  return ws + off + (size_t)side * 4 * sf_slot_len(L, l);
}

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
// Coefficient shift by z across the warp: lane j receives lane j - 1's value, lane 0 zero.
__device__ __forceinline__ double2 shfl_up2(double2 v, int lane) {
  const double2 u = make_double2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
  return lane == 0 ? make_double2(0.0, 0.0) : u;
}

// Leaf: the s <= 32 Schur steps of a node on its windows (its first coefficient at index a of
// Phi and Psi), accumulating Theta from the identity. Run by one whole warp; returns false (in every lane) if a pivot 1 - |eps|^2 is not
// positive. out: four polynomials (Theta_00, Theta_01, Theta_10, Theta_11) of stride len >= s + 1.
// The windows and results are written by this CTA during the launch: plain (coherent) loads.
__device__ bool sf_leaf(const double2* Phi, const double2* Psi, int a, int s, double2* out, int len, int lane) {
  const double2 zero = make_double2(0.0, 0.0);
  double2 ph = lane < s ? Phi[a + lane] : zero;
  double2 ps = lane < s ? Psi[a + lane] : zero;
  double2 t00 = lane == 0 ? make_double2(1.0, 0.0) : zero, t01 = zero, t10 = zero, t11 = t00;
  double2 top01 = zero, top11 = zero;  // coefficient 32 of column 1 (only after a 32nd step)
  for (int t = 0; t < s; ++t) {
    const double2 pt = shfl2(ph, t), st = shfl2(ps, t);
    const double sn = st.x * st.x + st.y * st.y;
    if (!(sn > 0.0)) return false;
    const double2 eps = make_double2((pt.x * st.x + pt.y * st.y) / sn, (pt.y * st.x - pt.x * st.y) / sn);
    const double den = 1.0 - (eps.x * eps.x + eps.y * eps.y);
    if (!(den > 1e-300)) return false;
    const double inv = 1.0 / den;
    const double2 ec = cconj(eps);
    const double2 nph = cscale(csub(ph, cmul(eps, ps)), inv);
    const double2 cps = cscale(csub(ps, cmul(ec, ph)), inv);
    const double2 n00 = cscale(csub(t00, cmul(eps, t01)), inv);
    const double2 n10 = cscale(csub(t10, cmul(eps, t11)), inv);
    const double2 c01 = cscale(csub(t01, cmul(ec, t00)), inv);
    const double2 c11 = cscale(csub(t11, cmul(ec, t10)), inv);
    ph = nph;
    t00 = n00;
    t10 = n10;
    ps = shfl_up2(cps, lane);
    t01 = shfl_up2(c01, lane);
    t11 = shfl_up2(c11, lane);
    top01 = shfl2(c01, 31);
    top11 = shfl2(c11, 31);
  }
  if (lane <= s) {
    out[lane] = t00;
    out[len + lane] = t01;
    out[2 * len + lane] = t10;
    out[3 * len + lane] = t11;
  }
  if (s == 32 && lane == 0) {
    out[32] = zero;
    out[len + 32] = top01;
    out[2 * len + 32] = zero;
    out[3 * len + 32] = top11;
  }
  return true;
}

template <int P> struct sf_shape {
  static constexpr int E = P >= 512 ? P / 256 : 2;
  static constexpr int T = P / E;
};

// Window map of a node of s steps (first coefficient at index a of Phi, Psi) with a left child of
// s1 steps: [phi, psi] Theta_left on the node's coefficients s1 .. s - 1, written to the right
// child's windows PhiR, PsiR from index 0. T1: the left child's four polynomials (n1 = s1 + 1
// coefficients, stride len1). Shared memory: 2P exchange + 3P held spectra.
// MINB only separates the copies compiled for the two register budgets of k_superfast.
template <int P, int MINB>
__device__ __noinline__ void sf_update(const double2* Phi, const double2* Psi, int a, int s, int s1,
                                       const double2* T1, int len1, double2* PhiR, double2* PsiR, double2* smem,
                                       const double2* __restrict__ tw, int t) {
  constexpr int E = sf_shape<P>::E, T = sf_shape<P>::T;
  if (t >= T) return;
  const double2 zero = make_double2(0.0, 0.0);
  double2* ex = smem;
  double2* H = smem + 2 * P;
  const int n1 = s1 + 1;
  double2 v[2][E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    v[0][r] = i < s ? Phi[a + i] : zero;
    v[1][r] = i < s ? Psi[a + i] : zero;
  }
  block_fft<P, E, 2, -1>(v, ex, tw, t, 1);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    H[t + T * r] = v[0][r];
    H[P + t + T * r] = v[1][r];
  }
#pragma unroll
  for (int r = 0; r < E; ++r) {  // column 0 of Theta_{a,m}: Theta_00, Theta_10
    const int i = t + T * r;
    v[0][r] = i < n1 ? T1[i] : zero;
    v[1][r] = i < n1 ? T1[2 * len1 + i] : zero;
  }
  block_fft<P, E, 2, -1>(v, ex, tw, t, 1);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    H[2 * P + i] = cadd(cmul(H[i], v[0][r]), cmul(H[P + i], v[1][r]));
  }
#pragma unroll
  for (int r = 0; r < E; ++r) {  // column 1: Theta_01, Theta_11
    const int i = t + T * r;
    v[0][r] = i < n1 ? T1[len1 + i] : zero;
    v[1][r] = i < n1 ? T1[3 * len1 + i] : zero;
  }
  block_fft<P, E, 2, -1>(v, ex, tw, t, 1);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    const double2 q = cadd(cmul(H[i], v[0][r]), cmul(H[P + i], v[1][r]));
    v[0][r] = H[2 * P + i];
    v[1][r] = q;
  }
  block_fft<P, E, 2, +1>(v, ex, tw, t, 1);
  const double sc = 1.0 / P;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = t + T * r;
    if (i >= s1 && i < s) {
      PhiR[i - s1] = cscale(v[0][r], sc);
      PsiR[i - s1] = cscale(v[1][r], sc);
    }
  }
}

// Product Theta = T1 T2 of a node of s steps (children of s1 and s - s1 steps; n1, n2 coefficients,
// strides len1, len2), written with s + 1 coefficients at stride len. Shared memory: 2P exchange +
// 4P held spectra of T2. P >= s; when P == s the circular product wraps only the degree-s
// coefficient of column 1, onto its (zero) constant term.
template <int P, int MINB>
__device__ __noinline__ void sf_product(const double2* T1, int n1, int len1, const double2* T2, int n2, int len2, double2* out,
                           int len, int s, double2* smem, const double2* __restrict__ tw, int t) {
  constexpr int E = sf_shape<P>::E, T = sf_shape<P>::T;
  if (t >= T) return;
  const double2 zero = make_double2(0.0, 0.0);
  double2* ex = smem;
  double2* H = smem + 2 * P;
  double2 v[2][E];
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // h = 0: T2_00, T2_10 -> H0, H1; h = 1: T2_01, T2_11 -> H2, H3
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = t + T * r;
      v[0][r] = i < n2 ? T2[h * len2 + i] : zero;
      v[1][r] = i < n2 ? T2[(2 + h) * len2 + i] : zero;
    }
    block_fft<P, E, 2, -1>(v, ex, tw, t, 1);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      H[(2 * h) * P + t + T * r] = v[0][r];
      H[(2 * h + 1) * P + t + T * r] = v[1][r];
    }
  }
  const double sc = 1.0 / P;
#pragma unroll
  for (int row = 0; row < 2; ++row) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = t + T * r;
      v[0][r] = i < n1 ? T1[(2 * row) * len1 + i] : zero;
      v[1][r] = i < n1 ? T1[(2 * row + 1) * len1 + i] : zero;
    }
    block_fft<P, E, 2, -1>(v, ex, tw, t, 1);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = t + T * r;
      const double2 x0 = v[0][r], x1 = v[1][r];
      v[0][r] = cadd(cmul(x0, H[i]), cmul(x1, H[P + i]));
      v[1][r] = cadd(cmul(x0, H[2 * P + i]), cmul(x1, H[3 * P + i]));
    }
    block_fft<P, E, 2, +1>(v, ex, tw, t, 1);
    double2* o0 = out + (2 * row) * len;
    double2* o1 = out + (2 * row + 1) * len;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = t + T * r;
      const double2 c0 = cscale(v[0][r], sc), c1 = cscale(v[1][r], sc);
      if (i <= s) o0[i] = c0;
      if (P == s) {
        if (i == 0) {
          o0[s] = zero;
          o1[0] = zero;
          o1[s] = c1;
        } else {
          o1[i] = c1;
        }
      } else if (i <= s) {
        o1[i] = c1;
      }
    }
  }
}

template <int MINB>
__device__ void sf_update_any(int P, const double2* Phi, const double2* Psi, int a, int s, int s1, const double2* T1,
                              int len1, double2* PhiR, double2* PsiR, double2* smem, const double2* tw, int t) {
  switch (P) {
    case 64: sf_update<64, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
    case 128: sf_update<128, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
    case 256: sf_update<256, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
    case 512: sf_update<512, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
    case 1024: sf_update<1024, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
    default: sf_update<2048, MINB>(Phi, Psi, a, s, s1, T1, len1, PhiR, PsiR, smem, tw, t); break;
  }
}

template <int MINB>
__device__ void sf_product_any(int P, const double2* T1, int n1, int len1, const double2* T2, int n2, int len2,
                               double2* out, int len, int s, double2* smem, const double2* tw, int t) {
  switch (P) {
    case 64: sf_product<64, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
    case 128: sf_product<128, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
    case 256: sf_product<256, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
    case 512: sf_product<512, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
    case 1024: sf_product<1024, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
    default: sf_product<2048, MINB>(T1, n1, len1, T2, n2, len2, out, len, s, smem, tw, t); break;
  }
}

// A node [a, b) of the recursion: phase 0 (left child next), 1 (window map, then right child),
// 2 (product); side 0/1 for a left/right child; its windows in the buffer of depth wb, whose
// index 0 holds coefficient wbase.
struct sf_frame {
  int a, b, phase, side, wb, wbase;
};

// gen: [count][L] generators a(d) (first column c[d] = conj(a(d))); x: [count][L]; ws: gridDim.x
// slots of ws_elems. Writes FBST_ERR_NUMERIC to *status if a pivot is not positive.
// MINB: resident CTAs per SM the register budget is cut for (2 up to L = 1025, whose FFTs of at
// most 1024 points need 96 KB of shared memory; 1 beyond, where 192 KB allow one CTA per SM anyway
// and the 2048-point products get the registers they need).
template <int MINB>
__global__ void __launch_bounds__(kSfThreads, MINB)
    k_superfast(const double2* __restrict__ gen, double2* __restrict__ xout, int L, int count, double2* ws_all,
                size_t ws_elems, const double2* __restrict__ tw, int* status) {
  extern __shared__ double2 sf_smem[];
  __shared__ int bad;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  double2* ws = ws_all + (size_t)blockIdx.x * ws_elems;
  double2* Phi = ws;  // depth-0 windows, indexed by coefficient
  double2* Psi = ws + L;
  for (int sys = blockIdx.x; sys < count; sys += gridDim.x) {
    const double2* g = gen + (size_t)sys * L;
    double2* x = xout + (size_t)sys * L;
    const double c0 = g[0].x;
    if (!(c0 > 0.0)) {  // uniform: every thread reads the same value
      if (t == 0) atomicExch(status, (int)FBST_ERR_NUMERIC);
      continue;
    }
    if (L == 1) {
      if (t == 0) x[0] = make_double2(1.0 / c0, 0.0);
      continue;
    }
    const double ic0 = 1.0 / c0;
    for (int k = 1 + t; k < L; k += blockDim.x) {
      Phi[k] = cscale(cconj(g[k]), ic0);      // phi_1 = c / c[0]
      Psi[k] = cscale(cconj(g[k - 1]), ic0);  // psi_1 = z c / c[0]
    }
    if (t == 0) bad = 0;
    __syncthreads();
    sf_frame st[kSfMaxDepth + 1];
    int top = 0;
    st[0] = sf_frame{1, L, 0, 0, 0, 0};
    while (top >= 0) {
      const sf_frame f = st[top];
      const int s = f.b - f.a, l = top;
      double2* out = sf_slot(ws, L, l, f.side);
      const int len = sf_slot_len(L, l);
      const double2* Wphi = ws + sf_win_off(L, f.wb);
      const double2* Wpsi = Wphi + sf_win_len(L, f.wb);
      const int ar = f.a - f.wbase;
      if (s <= kSfLeaf) {
        if (warp == 0 && !sf_leaf(Wphi, Wpsi, ar, s, out, len, lane) && lane == 0) bad = 1;
        __syncthreads();
        if (bad) break;
        --top;
        continue;
      }
      const int m = f.a + s / 2, s1 = m - f.a;
      int P = 64;
      while (P < s) P *= 2;
      const double2* T1 = sf_slot(ws, L, l + 1, 0);
      const int len1 = sf_slot_len(L, l + 1);
      if (f.phase == 0) {
        st[top].phase = 1;
        st[++top] = sf_frame{f.a, m, 0, 0, f.wb, f.wbase};
      } else if (f.phase == 1) {
        double2* Rphi = ws + sf_win_off(L, l + 1);
        sf_update_any<MINB>(P, Wphi, Wpsi, ar, s, s1, T1, len1, Rphi, Rphi + sf_win_len(L, l + 1), sf_smem, tw, t);
        __syncthreads();
        st[top].phase = 2;
        st[++top] = sf_frame{m, f.b, 0, 1, l + 1, m};
      } else {
        sf_product_any<MINB>(P, T1, s1 + 1, len1, sf_slot(ws, L, l + 1, 1), s - s1 + 1, len1, out, len, s, sf_smem, tw, t);
        __syncthreads();
        --top;
      }
    }
    if (bad) {
      if (t == 0) atomicExch(status, (int)FBST_ERR_NUMERIC);
      __syncthreads();
      continue;
    }
    // x = f_L = (Theta_00 + z Theta_10) / c[0], Theta at depth 0 (L coefficients suffice).
    const double2* th = sf_slot(ws, L, 0, 0);
    const int len0 = sf_slot_len(L, 0);
    for (int k = t; k < L; k += blockDim.x) {
      double2 v = th[k];
      if (k >= 1) v = cadd(v, th[2 * len0 + k - 1]);
      x[k] = cscale(v, ic0);
    }
    __syncthreads();
  }
}

}  // namespace

size_t superfast_smem_bytes(int L) {
  if (L - 1 <= kSfLeaf) return 0;
  int P = 64;
  while (P < L - 1) P *= 2;
  return 6 * (size_t)P * sizeof(double2);
}

int solve_generators(fbst_plan_s* p, const double2* gen, double2* x, int count, int method, cudaStream_t s) {
  const int L = p->info.L;
  if (count <= 0) return FBST_OK;
  if (method == FBST_GEN_LEVINSON) return launch_levinson(gen, x, count, L, p->d_status, s);
  if (method != FBST_GEN_SUPERFAST) return FBST_ERR_INVALID;
  if (L - 1 > 2048 || sf_depth(L) > kSfMaxDepth) return FBST_ERR_UNSUPPORTED;
  const size_t smem = superfast_smem_bytes(L);
  // The largest dynamic shared memory each form needs (P = 1024 and P = 2048), below the 227 KB
  // opt-in limit less the kernel's static shared word.
  static const cudaError_t attr2 = cudaFuncSetAttribute(k_superfast<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)superfast_smem_bytes(1025));
  static const cudaError_t attr1 = cudaFuncSetAttribute(k_superfast<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        (int)superfast_smem_bytes(2049));
  const bool big = L - 1 > 1024;
  FBST_CUDA_TRY(big ? attr1 : attr2);
  const int ctas = grid_for_items(count, big ? resident_ctas(k_superfast<1>, kSfThreads, smem)
                                             : resident_ctas(k_superfast<2>, kSfThreads, smem));
  const size_t elems = sf_ws_elems(L);
  double2* ws = nullptr;
  FBST_TRY(plan_alloc_n(p, &ws, (size_t)ctas * elems));
  // The workspace is allocated and freed in stream order on the plan's stream; on another stream
  // the launch waits for the allocation and the free for the launch.
  const bool other = s != p->mem_stream;
  cudaError_t e = other ? cudaStreamSynchronize(p->mem_stream) : cudaSuccess;
  if (e == cudaSuccess) {
    if (big) k_superfast<1><<<ctas, kSfThreads, smem, s>>>(gen, x, L, count, ws, elems, p->tw64, p->d_status);
    else k_superfast<2><<<ctas, kSfThreads, smem, s>>>(gen, x, L, count, ws, elems, p->tw64, p->d_status);
    e = cudaGetLastError();
  }
  if (other) cudaStreamSynchronize(s);
  plan_free(p, ws);
  FBST_CUDA_TRY(e);
  return FBST_OK;
}

}  // namespace fbst
