// Self single-layer matrix S (2N x 2N) of every vesicle (Eqs. single_layer, Stokeslet; Sec. 2.2.2).
//
// S_ab[i][j] = sa_j/(4 pi mu) * ( delta_ab * lp_ij + (2 pi/N) * rr_ab_ij ) with
//   lp_ij = -R(i-j)/2 - (pi/N) log(|r_ij|^2 / (4 sin^2(pi (i-j)/N)))    (i != j)
//   lp_ii = -R(0)/2 - (2 pi/N) log(sa_i)
//   rr_ij = r r^T / |r|^2 (i != j),  rr_ii = X_s X_s^T
// i.e. the Kress product rule for the log singularity of -log|r| and the trapezoid rule for the
// smooth remainder, with the standard 2D Stokeslet (1/4 pi mu)(-log|r| I + r r^T/|r|^2).
// Row-major, rows [x-velocity(0..N-1), y-velocity(0..N-1)], columns [f_x, f_y].
#pragma once
#include "common.cuh"

namespace vs {

__global__ void __launch_bounds__(256) k_self_matrix(VesIndex vi, const double* __restrict__ xy,
                                                     const double* __restrict__ sa,
                                                     const double* __restrict__ tx,
                                                     const double* __restrict__ ty,
                                                     const double* __restrict__ tab, double mu,
                                                     double* __restrict__ scratch, int slot,
                                                     const int* __restrict__ active) {
  const int v = blockIdx.y;
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N * N) return;
  const int i = p / N, j = p - (p / N) * N;
  const int64_t o = vi.off[v];
  const double* T = tab + vi.toff[v];
  const int m = (i - j < 0) ? i - j + N : i - j;
  const double R = T[N + m];
  const double dal = 2.0 * VS_PI / N;
  double lp, axx, axy, ayy;
  if (i != j) {
    const double rx = xy[2 * o + i] - xy[2 * o + j];
    const double ry = xy[2 * o + N + i] - xy[2 * o + N + j];
    const double r2 = rx * rx + ry * ry;
    lp = -0.5 * R - 0.5 * dal * log(r2 / T[2 * N + m]);
    const double ir2 = 1.0 / r2;
    axx = rx * rx * ir2;
    axy = rx * ry * ir2;
    ayy = ry * ry * ir2;
  } else {
    lp = -0.5 * R - dal * log(sa[o + i]);
    const double a = tx[o + i], b = ty[o + i];
    axx = a * a;
    axy = a * b;
    ayy = b * b;
  }
  const double c = sa[o + j] / (4.0 * VS_PI * mu);
  double* S = scratch + vi.moff[v] + (MatLayout::slot(slot) + MatLayout::S) * (int64_t)N * N;
  const int n2 = 2 * N;
  S[(int64_t)i * n2 + j] = c * (lp + dal * axx);
  S[(int64_t)i * n2 + N + j] = c * dal * axy;
  S[(int64_t)(N + i) * n2 + j] = c * dal * axy;
  S[(int64_t)(N + i) * n2 + N + j] = c * (lp + dal * ayy);
}

}  // namespace vs
