// Host-built FP64 tables that depend only on the points per vesicle N (Sec. 2.2.1-2.2.2, 4.2).
//
// Layout for one N (TAB_STRIDE * N doubles):
//   [0,   N)  d(m)   first column of the Fourier differentiation circulant with the Nyquist
//                    mode dropped: d(0) = 0, d(m) = (-1)^m cot(pi m / N) / 2.
//   [N,  2N)  R(m)   Kress product-rule weights of log(4 sin^2((t - tau)/2)), N = 2n:
//                    R(m) = -(2 pi/n) sum_{k=1}^{n-1} cos(k t_m)/k - (pi/n^2) cos(n t_m), t_m = 2 pi m/N
//   [2N, 3N)  4 sin^2(pi m / N)
//   [3N, 9N)  K0(q)  interpolation kernel on the 6x finer grid, theta_q = 2 pi q/(6N):
//                    K0 = (1/N)[1 + 2 sum_{k=1}^{N/2-1} cos(k theta) + cos(N theta/2)]
//   [9N,15N)  K1(q)  its derivative in theta.
//   [15N,16N) cos(2 pi m / N),  [16N,17N) sin(2 pi m / N).
//   [17N,18N) -R(m)/2 + (pi/N) log(4 sin^2(pi m / N)) (m >= 1; 0 at m = 0): with it the log part of the
//             self single layer off the diagonal is this minus (pi/N) log|r|^2.
#pragma once
#include <cmath>
#include <vector>

namespace vs {

inline void build_tables(int N, double* t) {
  const int n = N / 2;
  for (int m = 0; m < N; ++m) {
    t[m] = (m == 0) ? 0.0 : 0.5 * ((m & 1) ? -1.0 : 1.0) / std::tan(VS_PI * m / N);
    const double tm = 2.0 * VS_PI * m / N;
    double R = 0.0;
    for (int k = 1; k < n; ++k) R -= (2.0 * VS_PI / n) * std::cos(k * tm) / k;
    R -= (VS_PI / ((double)n * n)) * std::cos(n * tm);
    t[N + m] = R;
    const double s = std::sin(VS_PI * m / N);
    t[2 * N + m] = 4.0 * s * s;
  }
  const int Nu = 6 * N;
  for (int q = 0; q < Nu; ++q) {
    const double th = 2.0 * VS_PI * q / Nu;
    double k0 = 1.0, k1 = 0.0;
    for (int k = 1; k < n; ++k) {
      k0 += 2.0 * std::cos(k * th);
      k1 -= 2.0 * k * std::sin(k * th);
    }
    k0 += std::cos(n * th);
    k1 -= n * std::sin(n * th);
    t[3 * N + q] = k0 / N;
    t[9 * N + q] = k1 / N;
  }
  for (int m = 0; m < N; ++m) {
    t[15 * N + m] = std::cos(2.0 * VS_PI * m / N);
    t[16 * N + m] = std::sin(2.0 * VS_PI * m / N);
    t[17 * N + m] = (m == 0) ? 0.0 : -0.5 * t[N + m] + (VS_PI / N) * std::log(t[2 * N + m]);
  }
}

}  // namespace vs
