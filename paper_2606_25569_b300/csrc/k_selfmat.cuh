// Self single-layer matrix S (2N x 2N) of every vesicle (Eqs. single_layer, Stokeslet; Sec. 2.2.2).
//
// S_ab[i][j] = sa_j/(4 pi mu) * ( delta_ab * lp_ij + (2 pi/N) * rr_ab_ij ) with
//   lp_ij = -R(i-j)/2 - (pi/N) log(|r_ij|^2 / (4 sin^2(pi (i-j)/N)))    (i != j)
//   lp_ii = -R(0)/2 - (2 pi/N) log(sa_i)
//   rr_ij = r r^T / |r|^2 (i != j),  rr_ii = X_s X_s^T
// i.e. the Kress product rule for the log singularity of -log|r| and the trapezoid rule for the
// smooth remainder, with the standard 2D Stokeslet (1/4 pi mu)(-log|r| I + r r^T/|r|^2).
// Row-major, rows [x-velocity(0..N-1), y-velocity(0..N-1)], columns [f_x, f_y]. k_self_matrix writes
// FP64 S; k_self_matrix_df writes the split S = S_hi + S_lo (two FP32 matrices, the S and SL blocks of
// the FP32 scratch) for the mixed-precision path, entirely in double-float.
#pragma once
#include "common.cuh"
#include "dfloat.cuh"

namespace vs {

// The kernel of S is symmetric in (i, j) apart from the column factor sa_j, so each CTA evaluates
// one 16 x 16 tile (bi <= bj) of the symmetric part (the FP64 logarithm dominates the cost) and
// writes the tile and its mirror image (bj, bi). Grid: (nt (nt + 1) / 2, M), nt = ceil(N / 16).
constexpr int SM_TILE = 16;

__device__ __forceinline__ void self_store(double* S, int n2, int N, int i, int j, double c, double lp, double dal,
                                           double axx, double axy, double ayy) {
  const double sxx = c * (lp + dal * axx), sxy = c * dal * axy, syy = c * (lp + dal * ayy);
  S[(int64_t)i * n2 + j] = sxx;
  S[(int64_t)i * n2 + N + j] = sxy;
  S[(int64_t)(N + i) * n2 + j] = sxy;
  S[(int64_t)(N + i) * n2 + N + j] = syy;
}

__global__ void __launch_bounds__(256) k_self_matrix(VesIndex vi, const double* __restrict__ xy,
                                                     const double* __restrict__ sa,
                                                     const double* __restrict__ tx,
                                                     const double* __restrict__ ty,
                                                     const double* __restrict__ tab, double mu,
                                                     double* __restrict__ scratch, int slot,
                                                     const int* __restrict__ active) {
  const int v = vi.vid(blockIdx.y);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int nt = (N + SM_TILE - 1) / SM_TILE;
  int t = blockIdx.x, bi = 0;
  if (t >= nt * (nt + 1) / 2) return;
  while (t >= nt - bi) { t -= nt - bi; ++bi; }
  const int bj = bi + t;
  __shared__ double kl[SM_TILE][SM_TILE + 1], kxx[SM_TILE][SM_TILE + 1], kxy[SM_TILE][SM_TILE + 1],
      kyy[SM_TILE][SM_TILE + 1];
  const int li = threadIdx.x / SM_TILE, lj = threadIdx.x % SM_TILE;
  const int64_t o = vi.off[v];
  const double* T = tab + vi.toff[v];
  const double dal = 2.0 * VS_PI / N;
  const double c0 = 1.0 / (4.0 * VS_PI * mu);
  double* S = scratch + vi.moff[v] + (MatLayout::slot(slot) + MatLayout::S) * (int64_t)N * N;
  const int n2 = 2 * N;
  int i = bi * SM_TILE + li, j = bj * SM_TILE + lj;
  if (i < N && j < N) {
    const int m = (i - j < 0) ? i - j + N : i - j;
    const double R = T[N + m];
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
    kl[li][lj] = lp;
    kxx[li][lj] = axx;
    kxy[li][lj] = axy;
    kyy[li][lj] = ayy;
    self_store(S, n2, N, i, j, sa[o + j] * c0, lp, dal, axx, axy, ayy);
  }
  if (bi == bj) return;
  __syncthreads();
  // mirror tile: entry (i, j) = (bj*16 + li, bi*16 + lj) has the symmetric part of (j, i)
  i = bj * SM_TILE + li;
  j = bi * SM_TILE + lj;
  if (i < N && j < N)
    self_store(S, n2, N, i, j, sa[o + j] * c0, kl[lj][li], dal, kxx[lj][li], kxy[lj][li], kyy[lj][li]);
}


__device__ __forceinline__ void self_store_df(float* Sh, float* Sl, int n2, int N, int i, int j, float2 c, float2 lp,
                                              float2 dal, float2 axx, float2 axy, float2 ayy) {
  const float2 sxx = df_mul(c, df_add(lp, df_mul(dal, axx)));
  const float2 sxy = df_mul(c, df_mul(dal, axy));
  const float2 syy = df_mul(c, df_add(lp, df_mul(dal, ayy)));
  const int64_t e0 = (int64_t)i * n2 + j, e1 = (int64_t)i * n2 + N + j, e2 = (int64_t)(N + i) * n2 + j,
                e3 = (int64_t)(N + i) * n2 + N + j;
  Sh[e0] = sxx.x; Sl[e0] = sxx.y;
  Sh[e1] = sxy.x; Sl[e1] = sxy.y;
  Sh[e2] = sxy.x; Sl[e2] = sxy.y;
  Sh[e3] = syy.x; Sl[e3] = syy.y;
}

// The same matrix as k_self_matrix, as S_hi + S_lo, entirely in double-float: log|r|^2 by log_df minus the
// tabulated log 4 sin^2, the r r^T/|r|^2 terms and the products. The per-point inputs (positions relative
// to point 0, weights |X_alpha|/(4 pi mu), the diagonal log term and the tangents) come as double-float
// pairs from k_geometry and the table in double-float, so no FP64 arithmetic is left here. Same grid and
// tiling as k_self_matrix.
__global__ void __launch_bounds__(256) k_self_matrix_df(VesIndex vi, const float4* __restrict__ sdf,
                                                        const float2* __restrict__ tabdf,
                                                        const float4* __restrict__ logtab,
                                                        float* __restrict__ scratch32, int slot,
                                                        const int* __restrict__ active) {
  const int v = vi.vid(blockIdx.y);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int nt = (N + SM_TILE - 1) / SM_TILE;
  int t = blockIdx.x, bi = 0;
  if (t >= nt * (nt + 1) / 2) return;
  while (t >= nt - bi) { t -= nt - bi; ++bi; }
  const int bj = bi + t;
  __shared__ float2 kl[SM_TILE][SM_TILE + 1], kxx[SM_TILE][SM_TILE + 1], kxy[SM_TILE][SM_TILE + 1],
      kyy[SM_TILE][SM_TILE + 1];
  __shared__ float2 cc[2][SM_TILE];     // |X_alpha|_j / (4 pi mu) for the tile's columns (0) and its mirror's (1)
  __shared__ float4 pr[2][SM_TILE];     // [rows, cols]: points of the tile relative to point 0 (x, y pairs)
  __shared__ float4 lt[LOG_TAB];
  __shared__ float2 am[2 * SM_TILE];  // the table's log constant at m = (bi - bj) 16 + d, d = -15..16
  __shared__ float2 kc[2];            // 2 pi / N and -pi / N in double-float
  for (int e = threadIdx.x; e < LOG_TAB; e += blockDim.x) lt[e] = logtab[e];
  const int li = threadIdx.x / SM_TILE, lj = threadIdx.x % SM_TILE;
  const int64_t o = vi.off[v];
  const float4* P = sdf + 3 * o;
  if (threadIdx.x < 2 * SM_TILE) {
    const int w = threadIdx.x / SM_TILE, l = threadIdx.x % SM_TILE;
    const int jj = (w ? bi : bj) * SM_TILE + l, k = (w ? bj : bi) * SM_TILE + l;
    cc[w][l] = (jj < N) ? make_float2(P[3 * jj + 1].x, P[3 * jj + 1].y) : make_float2(0.f, 0.f);
    pr[w][l] = (k < N) ? P[3 * k] : make_float4(0.f, 0.f, 0.f, 0.f);
  } else if (threadIdx.x < 4 * SM_TILE) {
    const int d = threadIdx.x - 2 * SM_TILE - (SM_TILE - 1);
    int m = ((bi - bj) * SM_TILE + d) % N;
    if (m < 0) m += N;
    am[d + SM_TILE - 1] = tabdf[vi.toff[v] + 17 * N + m];
  } else if (threadIdx.x == 4 * SM_TILE) {
    const double dal64 = 2.0 * VS_PI / N;
    kc[0] = df_of(dal64);
    kc[1] = df_of(-0.5 * dal64);
  }
  __syncthreads();
  const float2 dal = kc[0];
  const int64_t NN = (int64_t)N * N;
  float* Sh = scratch32 + vi.moff[v] + (MatLayout::slot(slot) + MatLayout::S) * NN;
  float* Sl = scratch32 + vi.moff[v] + (MatLayout::slot(slot) + MatLayout::SL) * NN;
  const int n2 = 2 * N;
  int i = bi * SM_TILE + li, j = bj * SM_TILE + lj;
  float2 lp, axx, axy, ayy;
  const bool in = i < N && j < N;
  if (in) {
    if (i != j) {
      const float4 pi = pr[0][li], pj = pr[1][lj];
      const float2 rxd = df_add(make_float2(pi.x, pi.y), make_float2(-pj.x, -pj.y));
      const float2 ryd = df_add(make_float2(pi.z, pi.w), make_float2(-pj.z, -pj.w));
      const float2 xx = df_mul(rxd, rxd), xy2 = df_mul(rxd, ryd), yy = df_mul(ryd, ryd);
      const float2 r2 = df_add(xx, yy);
      lp = df_add(am[li - lj + SM_TILE - 1], df_mul(kc[1], log_df(r2, lt)));
      const float2 ir2 = df_rcp(r2);
      axx = df_mul(xx, ir2);
      axy = df_mul(xy2, ir2);
      ayy = df_mul(yy, ir2);
    } else {
      const float4 q = P[3 * i + 1], tg = P[3 * i + 2];
      lp = make_float2(q.z, q.w);
      const float2 a = make_float2(tg.x, tg.y), b = make_float2(tg.z, tg.w);
      axx = df_mul(a, a);
      axy = df_mul(a, b);
      ayy = df_mul(b, b);
    }
    kl[li][lj] = lp;
    kxx[li][lj] = axx;
    kxy[li][lj] = axy;
    kyy[li][lj] = ayy;
  }
  __syncthreads();
  if (in) self_store_df(Sh, Sl, n2, N, i, j, cc[0][lj], lp, dal, axx, axy, ayy);
  if (bi == bj) return;
  // mirror tile: entry (i, j) = (bj*16 + li, bi*16 + lj) has the symmetric part of (j, i)
  i = bj * SM_TILE + li;
  j = bi * SM_TILE + lj;
  if (i < N && j < N)
    self_store_df(Sh, Sl, n2, N, i, j, cc[1][lj], kl[lj][li], dal, kxx[lj][li], kxy[lj][li], kyy[lj][li]);
}

}  // namespace vs
