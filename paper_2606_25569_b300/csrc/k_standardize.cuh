// Standardisation for the networks (Sec. 3.4.1; Algorithms 2-4) and its inverse for displacements.
//
// k_standardize, one CTA (NMAX threads) per vesicle:
//   centre c = (2/3) int X (X.n) ds / int X.n ds (the area centroid; the printed ratio lacks 2/3),
//   J = 1/4 int (r.n)(|r|^2 I - r r^T) ds, principal axis = eigenvector of the smallest eigenvalue
//   (y component >= 0), rotation taking it to +y, scale 1/L, cyclic shift so that point 0 is the
//   right-most upward crossing of the x axis, then the Fourier filter (modes |k| <= kmax kept,
//   kmax < N/2, so the Nyquist mode is always removed).
//   Writes the frame parameters and either the filtered shape as an FP32 row [x^o(N), y^o(N)] or its
//   Fourier features (the network input, below).
// k_destandardize_add: X += R^T (out_scale * dX^o) / s, shifted back to the original labels, where
//   dX^o is synthesised from the network's Fourier features.
//
// Fourier features of a curve or displacement v^o (standard frame, relabelled), K = min(kmax, N/2 - 1):
//   a_k = (1/N) sum_j v_j cos(2 pi k j / N),  b_k = -(1/N) sum_j v_j sin(2 pi k j / N),
//   v_j = a_0 + 2 sum_{k=1..K} (a_k cos(2 pi k j / N) - b_k sin(2 pi k j / N))   (modes <= K),
// row = [a_0..a_K, b_1..b_K of x; a_0..a_K, b_1..b_K of y; zeros] of width feat_width(K) =
// 16 ceil((4K + 2) / 16). Per-feature normalisation of such rows puts every mode on the same footing:
// the modes that the bending force amplifies by k^4 are the smallest ones.
#pragma once
#include "common.cuh"

namespace vs {

__host__ __device__ constexpr int feat_count(int K) { return 4 * K + 2; }
__host__ __device__ constexpr int feat_width(int K) { return (feat_count(K) + 15) / 16 * 16; }
__host__ __device__ inline int feat_kmax(int kmax, int N) { return kmax < N / 2 - 1 ? kmax : N / 2 - 1; }

struct StdFrame {
  double cx, cy, ct, st, s;
  int j0;
  int pad;
};

// The feature row (modes 0..K of cre, cim) of one vesicle, padded with zeros to feat_width(K).
__device__ __forceinline__ void write_features(const double (*cre)[NMAX / 2], const double (*cim)[NMAX / 2], int K,
                                               float* row) {
  const int per = 2 * K + 1, w = feat_width(K);
  for (int e = threadIdx.x; e < w; e += blockDim.x) {
    double val = 0.0;
    if (e < 2 * per) {
      const int comp = e / per, r = e - comp * per;
      val = (r <= K) ? cre[comp][r] : cim[comp][r - K];
    }
    row[e] = (float)val;
  }
}

__global__ void __launch_bounds__(NMAX) k_standardize(VesIndex vi, const double* __restrict__ xy,
                                                      const double* __restrict__ tab, float* __restrict__ xin,
                                                      int64_t ld_in, StdFrame* __restrict__ frame, int kmax,
                                                      bool features) {
  __shared__ double d[NMAX], xs[NMAX], ys[NMAX], xr[NMAX], yr[NMAX], red[NMAX / 32];
  __shared__ double cre[2][NMAX / 2], cim[2][NMAX / 2];
  __shared__ int sj0;
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const bool act = i < N;
  const double* T = tab + vi.toff[v];
  if (act) {
    d[i] = T[i];
    xs[i] = xy[2 * o + i];
    ys[i] = xy[2 * o + N + i];
  }
  __syncthreads();
  double xa = 0.0, ya = 0.0;
  if (act) {
    xa = circ_row(d, xs, N, i);
    ya = circ_row(d, ys, N, i);
  }
  const double sa = act ? sqrt(xa * xa + ya * ya) : 1.0;
  const double nx = ya / sa, ny = -xa / sa;  // outward normal (t_y, -t_x)
  const double w = act ? sa * 2.0 * VS_PI / N : 0.0;
  const double X = act ? xs[i] : 0.0, Y = act ? ys[i] : 0.0;
  const double xn = X * nx + Y * ny;
  const double den = block_sum(xn * w, red);
  const double cx = block_sum(X * xn * w, red) / (1.5 * den);
  const double cy = block_sum(Y * xn * w, red) / (1.5 * den);
  const double L = block_sum(w, red);
  const double rx = X - cx, ry = Y - cy;
  const double rn = rx * nx + ry * ny, r2 = rx * rx + ry * ry;
  const double Ja = 0.25 * block_sum(rn * (r2 - rx * rx) * w, red);
  const double Jb = 0.25 * block_sum(rn * (-rx * ry) * w, red);
  const double Jd = 0.25 * block_sum(rn * (r2 - ry * ry) * w, red);
  // smallest eigenvalue and its eigenvector (the better conditioned of two equivalent forms)
  const double hm = 0.5 * (Ja + Jd), hd = 0.5 * (Ja - Jd);
  const double lam = hm - sqrt(hd * hd + Jb * Jb);
  double px = lam - Jd, py = Jb;
  const double qx = Jb, qy = lam - Ja;
  if (qx * qx + qy * qy > px * px + py * py) { px = qx; py = qy; }
  const double pn = sqrt(px * px + py * py);
  px /= pn;
  py /= pn;
  if (py < 0.0 || (py == 0.0 && px < 0.0)) { px = -px; py = -py; }
  const double ct = py, st = px, s = 1.0 / L;
  if (act) {
    xr[i] = s * (ct * rx - st * ry);
    yr[i] = s * (st * rx + ct * ry);
  }
  __syncthreads();
  // right-most upward crossing: y_{j-1} < 0 <= y_j (smallest index on ties)
  double best = -1e300;
  int bj = N;
  if (act) {
    const int jm = (i == 0) ? N - 1 : i - 1;
    if (yr[jm] < 0.0 && yr[i] >= 0.0) { best = xr[i]; bj = i; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
    if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
  }
  __shared__ double rb[NMAX / 32];
  __shared__ int rj[NMAX / 32];
  if ((i & 31) == 0) { rb[i >> 5] = best; rj[i >> 5] = bj; }
  __syncthreads();
  if (i == 0) {
    double b = rb[0];
    int j = rj[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
      if (rb[k] > b || (rb[k] == b && rj[k] < j)) { b = rb[k]; j = rj[k]; }
    sj0 = (j < N) ? j : 0;
  }
  __syncthreads();
  const int j0 = sj0;
  // Fourier coefficients k = 0..kmax of the shifted curve (kmax < N/2)
  const int nk = min(kmax, N / 2 - 1) + 1;
  for (int e = i; e < 2 * nk; e += blockDim.x) {
    const int comp = e / nk, k = e - comp * nk;
    const double* src = comp ? yr : xr;
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      const double val = src[(j + j0) % N];
      re = fma(val, T[15 * N + m], re);
      im = fma(-val, T[16 * N + m], im);
      m += k;
      if (m >= N) m -= N;
    }
    cre[comp][k] = re / N;
    cim[comp][k] = im / N;
  }
  __syncthreads();
  if (i == 0) frame[v] = StdFrame{cx, cy, ct, st, s, j0, 0};
  if (features) {
    write_features(cre, cim, nk - 1, xin + (int64_t)v * ld_in);
    return;
  }
  if (act) {
    double fx = cre[0][0], fy = cre[1][0];
    int m = 0;
    for (int k = 1; k < nk; ++k) {
      m += i;
      if (m >= N) m -= N;
      const double c = T[15 * N + m], sn = T[16 * N + m];
      fx += 2.0 * (cre[0][k] * c - cim[0][k] * sn);
      fy += 2.0 * (cre[1][k] * c - cim[1][k] * sn);
    }
    xin[(int64_t)v * ld_in + i] = (float)fx;
    xin[(int64_t)v * ld_in + N + i] = (float)fy;
  }
}

// xy[v] += R^T (scale * dX^o) / s with the labels shifted back by j0, dX^o synthesised at label k from
// the Fourier features of row v of yout (modes <= K).
__global__ void __launch_bounds__(NMAX) k_destandardize_add(VesIndex vi, const float* __restrict__ yout,
                                                            int64_t ld_out, double scale, int kmax,
                                                            const double* __restrict__ tab,
                                                            const StdFrame* __restrict__ frame,
                                                            double* __restrict__ xy) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int k = threadIdx.x;
  if (k >= N) return;
  const int K = feat_kmax(kmax, N), per = 2 * K + 1;
  const double* T = tab + vi.toff[v];
  const float* row = yout + (int64_t)v * ld_out;
  double dx = row[0], dy = row[per];
  int m = 0;
  for (int q = 1; q <= K; ++q) {
    m += k;
    if (m >= N) m -= N;
    const double c = T[15 * N + m], sn = T[16 * N + m];
    dx += 2.0 * ((double)row[q] * c - (double)row[K + q] * sn);
    dy += 2.0 * ((double)row[per + q] * c - (double)row[per + K + q] * sn);
  }
  const StdFrame f = frame[v];
  dx *= scale / f.s;
  dy *= scale / f.s;
  const int i = (k + f.j0) % N;
  xy[2 * o + i] += f.ct * dx + f.st * dy;
  xy[2 * o + N + i] += -f.st * dx + f.ct * dy;
}

// Training targets: the displacement X_out - X_in of each vesicle expressed in the standard frame of
// X_in (rotation, unit length, relabelling), divided by out_scale, as Fourier features (modes <= K).
__global__ void __launch_bounds__(NMAX) k_to_frame_rows(VesIndex vi, const double* __restrict__ xin,
                                                        const double* __restrict__ xout,
                                                        const StdFrame* __restrict__ frame, double inv_scale,
                                                        const double* __restrict__ tab, int kmax,
                                                        float* __restrict__ rows, int64_t ld) {
  __shared__ double d[2][NMAX];
  __shared__ double cre[2][NMAX / 2], cim[2][NMAX / 2];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int k = threadIdx.x;
  const StdFrame f = frame[v];
  const double* T = tab + vi.toff[v];
  if (k < N) {
    const int i = (k + f.j0) % N;
    const double dx = xout[2 * o + i] - xin[2 * o + i], dy = xout[2 * o + N + i] - xin[2 * o + N + i];
    d[0][k] = f.s * (f.ct * dx - f.st * dy) * inv_scale;
    d[1][k] = f.s * (f.st * dx + f.ct * dy) * inv_scale;
  }
  __syncthreads();
  const int K = feat_kmax(kmax, N), nk = K + 1;
  for (int e = k; e < 2 * nk; e += blockDim.x) {
    const int comp = e / nk, q = e - comp * nk;
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(d[comp][j], T[15 * N + m], re);
      im = fma(-d[comp][j], T[16 * N + m], im);
      m += q;
      if (m >= N) m -= N;
    }
    cre[comp][q] = re / N;
    cim[comp][q] = im / N;
  }
  __syncthreads();
  write_features(cre, cim, K, rows + (int64_t)v * ld);
}

// Low-pass of each vesicle's points along the curve parameter: modes |k| > kmax (and the Nyquist
// mode) removed from x and y. The learned relaxation ends with it, so modes the network does not
// represent are not carried (the exact relaxation leaves them at their tiny size).
__global__ void __launch_bounds__(NMAX) k_lowpass(VesIndex vi, const double* __restrict__ tab, int kmax,
                                                  double* __restrict__ xy) {
  __shared__ double xs[NMAX], ys[NMAX];
  __shared__ double cre[2][NMAX / 2], cim[2][NMAX / 2];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const double* T = tab + vi.toff[v];
  if (i < N) {
    xs[i] = xy[2 * o + i];
    ys[i] = xy[2 * o + N + i];
  }
  __syncthreads();
  const int nk = min(kmax, N / 2 - 1) + 1;
  for (int e = i; e < 2 * nk; e += blockDim.x) {
    const int comp = e / nk, k = e - comp * nk;
    const double* src = comp ? ys : xs;
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(src[j], T[15 * N + m], re);
      im = fma(-src[j], T[16 * N + m], im);
      m += k;
      if (m >= N) m -= N;
    }
    cre[comp][k] = re / N;
    cim[comp][k] = im / N;
  }
  __syncthreads();
  if (i < N) {
    double fx = cre[0][0], fy = cre[1][0];
    int m = 0;
    for (int k = 1; k < nk; ++k) {
      m += i;
      if (m >= N) m -= N;
      const double c = T[15 * N + m], sn = T[16 * N + m];
      fx += 2.0 * (cre[0][k] * c - cim[0][k] * sn);
      fy += 2.0 * (cre[1][k] * c - cim[1][k] * sn);
    }
    xy[2 * o + i] = fx;
    xy[2 * o + N + i] = fy;
  }
}

}  // namespace vs
