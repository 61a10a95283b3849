// Learned advection and tension of the hybrid step (Sec. 3.2: Eqs. advectionMap, advTenMap and the
// self-tension map S_sigma; Table tab:networks), and the exact columns the networks are trained to.
//
// The interaction velocity u enters the advection X* = X^n + dt (I - M) u and the tension
// sigma = -L^{-1} P (B X + u) linearly. In each vesicle's standard frame (k_standardize: centred, principal
// axis along +y, unit length, point 0 on the positive x axis) u is expanded in the real Fourier modes
// k = 0..Kf of each component: with the features f of u (a_0..a_Kf, b_1..b_Kf of x, then of y, the
// convention of k_standardize), u = sum_i f_i psi_i for modes <= Kf, psi_i the field of one component equal
// to 1 (a_0), 2 cos(k alpha) (a_k) or -2 sin(k alpha) (b_k). The networks give, per vesicle, the columns
// (I - M) psi_i (velocity features up to Kout, 2 (2 Kout + 1) each), L^{-1} P psi_i and L^{-1} P B X (scalar
// features, 2 Kout + 1 each) of the standardised shape. (I - M) and L^{-1} P do not change with the
// vesicle's size; L^{-1} P B X of a vesicle of length L is that of its unit-length copy over L^2.
//
// Row layouts (FP32, one row per vesicle): advection  [column 0 | column 1 | ... ], CW = 2 (2 Kout + 1)
// floats per column; tension [S_sigma | column 0 | column 1 | ...], SW = 2 Kout + 1 floats each.
//
// Kernels (one CTA of NMAX threads per vesicle):
//   k_standard_points  the standardised points in FP64 (no filter), for building the exact columns;
//   k_basis_velocity   psi_i at every vesicle's points;
//   k_field_features   Fourier features (modes <= K) of a velocity or scalar field into a row at a column
//                      offset, optionally scaled and added to (the exact columns' assembly);
//   k_flow_apply       the learned advection (X* = X + dt R^T shift((sum_i f_i Q_i)(alpha))) or tension
//                      (sigma = -shift(S_sigma(alpha)) / L^2 - shift((sum_i f_i S_i)(alpha))).
#pragma once
#include "common.cuh"
#include "k_standardize.cuh"

namespace vs {

__host__ __device__ constexpr int flow_basis(int Kf) { return 4 * Kf + 2; }
__host__ __device__ constexpr int flow_col_adv(int Kout) { return 2 * (2 * Kout + 1); }
__host__ __device__ constexpr int flow_col_ten(int Kout) { return 2 * Kout + 1; }
__host__ __device__ constexpr int flow_adv_width(int Kf, int Kout) {
  return (flow_basis(Kf) * flow_col_adv(Kout) + 15) / 16 * 16;
}
__host__ __device__ constexpr int flow_ten_width(int Kf, int Kout) {
  return ((flow_basis(Kf) + 1) * flow_col_ten(Kout) + 15) / 16 * 16;
}

// The standardised points x^o_k = s R (X_{(k + j0) mod N} - c) in FP64, CSR blocks.
__global__ void __launch_bounds__(NMAX) k_standard_points(VesIndex vi, const double* __restrict__ xy,
                                                          const StdFrame* __restrict__ frame,
                                                          double* __restrict__ out) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int k = threadIdx.x;
  if (k >= N) return;
  const StdFrame f = frame[v];
  const int i = (k + f.j0) % N;
  const double rx = xy[2 * o + i] - f.cx, ry = xy[2 * o + N + i] - f.cy;
  out[2 * o + k] = f.s * (f.ct * rx - f.st * ry);
  out[2 * o + N + k] = f.s * (f.st * rx + f.ct * ry);
}

// psi_b (basis field b of Kf) at every vesicle's points, CSR blocks.
__global__ void __launch_bounds__(NMAX) k_basis_velocity(VesIndex vi, const double* __restrict__ tab, int b, int Kf,
                                                         double* __restrict__ u) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int j = threadIdx.x;
  if (j >= N) return;
  const double* T = tab + vi.toff[v];
  const int per = 2 * Kf + 1, comp = b / per, r = b - comp * per;
  double val;
  if (r == 0) {
    val = 1.0;
  } else if (r <= Kf) {
    val = 2.0 * T[15 * N + (r * j) % N];
  } else {
    val = -2.0 * T[16 * N + ((r - Kf) * j) % N];
  }
  u[2 * o + j] = comp == 0 ? val : 0.0;
  u[2 * o + N + j] = comp == 0 ? 0.0 : val;
}

// Row v, columns [col, col + (2K + 1) ncomp), of `rows` (+)= scale * features of the field: ncomp = 2, a
// velocity (CSR blocks, 2N per vesicle at 2 off); ncomp = 1, a scalar field (N per vesicle at off).
__global__ void __launch_bounds__(NMAX) k_field_features(VesIndex vi, const double* __restrict__ field, int ncomp,
                                                         const double* __restrict__ tab, int K, double scale,
                                                         bool add, float* __restrict__ rows, int64_t ld, int col) {
  __shared__ double d[2][NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int t = threadIdx.x;
  const double* T = tab + vi.toff[v];
  if (t < N)
    for (int c = 0; c < ncomp; ++c) d[c][t] = field[ncomp * o + c * N + t];
  __syncthreads();
  const int per = 2 * K + 1;
  float* row = rows + (int64_t)v * ld + col;
  for (int e = t; e < ncomp * per; e += blockDim.x) {
    const int c = e / per, r = e - c * per;
    const int q = r <= K ? r : r - K;
    const int off = r <= K ? 15 * N : 16 * N;
    double acc = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      acc = fma(d[c][j], T[off + m], acc);
      m += q;
      if (m >= N) m -= N;
    }
    const double val = (r <= K ? acc : -acc) / N * scale;
    row[e] = add ? (float)((double)row[e] + val) : (float)val;
  }
}

// Learned advection (ten == false): xo = xy + dt R^T shift(sum_i f_i Q_i); learned tension (ten == true):
// sigma = -shift(S_sigma) s^2 - shift(sum_i f_i S_i), s = 1/L of the frame. f = features (modes <= Kf) of
// the velocity u in the frame, the network row at rows + v ld.
template <bool TEN>
__global__ void __launch_bounds__(NMAX) k_flow_apply(VesIndex vi, const double* __restrict__ u,
                                                     const StdFrame* __restrict__ frame, const float* __restrict__ rows,
                                                     int64_t ld, int Kf, int Kout, const double* __restrict__ tab,
                                                     double dt, const double* __restrict__ xy, double* __restrict__ xo,
                                                     double* __restrict__ sigma) {
  __shared__ double w[2][NMAX];
  __shared__ double f[4 * (NMAX / 2) + 2];
  __shared__ double g[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int t = threadIdx.x;
  const double* T = tab + vi.toff[v];
  const StdFrame fr = frame[v];
  // u in the frame: rotated and relabelled (no scaling: the maps do not depend on the size)
  if (t < N) {
    const int i = (t + fr.j0) % N;
    const double ux = u[2 * o + i], uy = u[2 * o + N + i];
    w[0][t] = fr.ct * ux - fr.st * uy;
    w[1][t] = fr.st * ux + fr.ct * uy;
  }
  __syncthreads();
  const int pf = 2 * Kf + 1, nb = 2 * pf;
  for (int e = t; e < nb; e += blockDim.x) {
    const int c = e / pf, r = e - c * pf;
    const int q = r <= Kf ? r : r - Kf;
    const int off = r <= Kf ? 15 * N : 16 * N;
    double acc = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      acc = fma(w[c][j], T[off + m], acc);
      m += q;
      if (m >= N) m -= N;
    }
    f[e] = (r <= Kf ? acc : -acc) / N;
  }
  __syncthreads();
  // the combination of the columns, in features (modes <= Kout)
  const float* row = rows + (int64_t)v * ld;
  const int po = 2 * Kout + 1;
  const int cw = TEN ? po : 2 * po;
  const int base = TEN ? po : 0;
  const double ss = fr.s * fr.s;
  const double sgn = TEN ? -1.0 : 1.0;
  for (int e = t; e < cw; e += blockDim.x) {
    double acc = TEN ? -(double)row[e] * ss : 0.0;
    for (int i = 0; i < nb; ++i) acc = fma(sgn * f[i], (double)row[base + i * cw + e], acc);
    g[e] = acc;
  }
  __syncthreads();
  if (t >= N) return;
  // synthesis at label t of the frame, then back to the vesicle's own label i
  const int i = (t + fr.j0) % N;
  double a = g[0], b = TEN ? 0.0 : g[po];
  int m = 0;
  for (int q = 1; q <= Kout; ++q) {
    m += t;
    if (m >= N) m -= N;
    const double c = T[15 * N + m], sn = T[16 * N + m];
    a += 2.0 * (g[q] * c - g[Kout + q] * sn);
    if (!TEN) b += 2.0 * (g[po + q] * c - g[po + Kout + q] * sn);
  }
  if (TEN) {
    sigma[o + i] = a;
  } else {
    xo[2 * o + i] = xy[2 * o + i] + dt * (fr.ct * a + fr.st * b);
    xo[2 * o + N + i] = xy[2 * o + N + i] + dt * (-fr.st * a + fr.ct * b);
  }
}

}  // namespace vs
