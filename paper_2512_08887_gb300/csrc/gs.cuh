// Gohberg-Semencul application of A_b^{-1} (Sec. V).
//
// A_b is Hermitian positive-definite Toeplitz. With x = A_b^{-1} e_0 (first column, x_0 > 0 real)
// its last column is J conj(x) (A_b is persymmetric up to conjugation), and
//
//     A_b^{-1} = (1/x_0) [ L(x) L(x)^H - L(Z J conj(x)) L(Z J conj(x))^H ],
//
// where L(c) is the lower-triangular Toeplitz matrix with first column c, J reverses and Z shifts
// down by one. (The paper writes the formula as L_x U_y - L_y U_x without the 1/x_0 scale and the
// shift; this is the same identity with both made explicit.) Every triangular Toeplitz product is
// a linear convolution (L(c) u) or correlation (L(c)^H u) of length L, evaluated with a circulant
// of size P >= 2L-1: four forward/inverse FFT pairs in all, as the paper counts, of which the two
// correlations and the two convolutions share their transforms of w and of the sum.
//
// The plan stores Xs = FFT_P(x / sqrt(x_0)) / P and Vs = FFT_P(Z J conj(x) / sqrt(x_0)) / P, so the
// unnormalised inverse transforms below need no further scaling.
#pragma once

#include "fft.cuh"

namespace fbst {

// v (strided layout, w_b zero-padded to P) -> v = A_b^{-1} w_b in entries t + T*r < L.
// X, Vv: this thread's entries of Xs and Vs. sbuf: 2*fft_smem_elems<V>(P) elements.
template <int P, int E, typename V>
__device__ __forceinline__ void gs_apply(V (&v)[E], const V (&X)[E], const V (&Vv)[E], V* sbuf,
                                         const V* __restrict__ tw, int t, int L) {
  constexpr int T = P / E;
  V a[1][E];
#pragma unroll
  for (int r = 0; r < E; ++r) a[0][r] = v[r];
  block_fft<P, E, 1, -1>(a, sbuf, tw, t);             // W = FFT(w)
  V u[2][E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    u[0][r] = cmulc(a[0][r], X[r]);                    // correlation with x: L(x)^H w
    u[1][r] = cmulc(a[0][r], Vv[r]);                   // correlation with Z J conj(x)
  }
  block_fft<P, E, 2, +1>(u, sbuf, tw, t);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    if (t + T * r >= L) {                              // keep the first L entries only
      u[0][r] = V{0, 0};
      u[1][r] = V{0, 0};
    }
  }
  block_fft<P, E, 2, -1>(u, sbuf, tw, t);
#pragma unroll
  for (int r = 0; r < E; ++r) a[0][r] = csub(cmul(X[r], u[0][r]), cmul(Vv[r], u[1][r]));
  block_fft<P, E, 1, +1>(a, sbuf, tw, t);             // convolutions, summed in frequency
#pragma unroll
  for (int r = 0; r < E; ++r) v[r] = a[0][r];
}

}  // namespace fbst
