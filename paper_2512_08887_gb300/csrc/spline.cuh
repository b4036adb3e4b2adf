// Host-side interpolation weights shared by the off-grid beams (Sec. VIII-A) and the nulling of
// off-grid interferers (Sec. VIII-B): a natural cubic spline in the direction cosine through the K
// grid beams around a direction.
#pragma once

#include <algorithm>
#include <cmath>

namespace fbst {

constexpr int kMaxWindow = 16;

// Weights c (n of them) with s(xq) = sum_i c_i f_i for the natural cubic spline s through the
// points (x_i, f_i), x increasing: cubic between knots, continuous first and second derivatives
// at the inner knots, zero second derivative at both ends. For each unit data vector e_j the
// moments M_i = s''(x_i) solve the tridiagonal system
//   h_{i-1} M_{i-1} + 2 (h_{i-1} + h_i) M_i + h_i M_{i+1} = 6 (d_i - d_{i-1}),  M_0 = M_{n-1} = 0,
// with d_i = (f_{i+1} - f_i) / h_i (Thomas algorithm), and c_j = s_j(xq).
inline void spline_weights(const double* x, int n, double xq, double* c) {
  if (n == 1) {
    c[0] = 1.0;
    return;
  }
  double h[kMaxWindow], Mo[kMaxWindow], cp[kMaxWindow], dp[kMaxWindow];
  for (int i = 0; i + 1 < n; ++i) h[i] = x[i + 1] - x[i];
  int seg = 0;
  while (seg + 2 < n && xq >= x[seg + 1]) ++seg;
  const double a = x[seg + 1] - xq, b = xq - x[seg], hs = h[seg];
  for (int j = 0; j < n; ++j) {
    auto f = [j](int i) { return i == j ? 1.0 : 0.0; };
    for (int i = 0; i < n; ++i) Mo[i] = 0.0;
    const int m = n - 2;   // inner knots 1..n-2
    for (int r = 0; r < m; ++r) {
      const int i = r + 1;
      const double lo = r > 0 ? h[i - 1] : 0.0, di = 2.0 * (h[i - 1] + h[i]), up = r + 1 < m ? h[i] : 0.0;
      const double rhs = 6.0 * ((f(i + 1) - f(i)) / h[i] - (f(i) - f(i - 1)) / h[i - 1]);
      const double den = di - lo * (r > 0 ? cp[r - 1] : 0.0);
      cp[r] = up / den;
      dp[r] = (rhs - lo * (r > 0 ? dp[r - 1] : 0.0)) / den;
    }
    for (int r = m - 1; r >= 0; --r) Mo[r + 1] = dp[r] - (r + 1 < m ? cp[r] * Mo[r + 2] : 0.0);
    c[j] = (Mo[seg] * a * a * a + Mo[seg + 1] * b * b * b) / (6.0 * hs) + (f(seg) - Mo[seg] * hs * hs / 6.0) * a / hs +
           (f(seg + 1) - Mo[seg + 1] * hs * hs / 6.0) * b / hs;
  }
}

// First of the K consecutive grid indices (of nb) around the direction cosine c: K/2 on each side
// of the interval that holds it, moved inward at the ends of the grid.
inline int window_first(int nb, double c, int K) {
  const double coord = (c + 1.0) * nb / 2.0;   // grid index of c
  const int first = (int)std::floor(coord) - (K / 2 - 1);
  return std::min(std::max(first, 0), nb - K);
}

// Window start and spline weights of direction (u, v) on a grid of bx x by beams (by = 1 and
// ky = 1 for a linear array): weights along u (kx of them), then along v (ky), as floats.
inline void interp_terms(int bx, int by, bool two_axes, double u, double v, int kx, int ky, int* fx, int* fy,
                         float* w) {
  double x[kMaxWindow], c[kMaxWindow];
  *fx = window_first(bx, u, kx);
  for (int i = 0; i < kx; ++i) x[i] = -1.0 + 2.0 * (*fx + i) / bx;
  spline_weights(x, kx, u, c);
  for (int i = 0; i < kx; ++i) w[i] = (float)c[i];
  *fy = 0;
  if (two_axes) {
    *fy = window_first(by, v, ky);
    for (int j = 0; j < ky; ++j) x[j] = -1.0 + 2.0 * (*fy + j) / by;
    spline_weights(x, ky, v, c);
    for (int j = 0; j < ky; ++j) w[kx + j] = (float)c[j];
  } else {
    w[kx] = 1.0f;
  }
}

}  // namespace fbst
