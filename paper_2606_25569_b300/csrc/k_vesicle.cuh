// Per-vesicle step kernels: advection, relaxation solve, redistribution, tension, correction
// (Eqs. advection_disc, relaxation_disc, tension_disc; Sec. 4.2, 4.3). One CTA per vesicle.
#pragma once
#include "common.cuh"
#include "k_dense.cuh"

namespace vs {

struct PointGeom {
  const double* sa;
  const double* tx;
  const double* ty;
};

// X* = X^n + dt (u - T L^{-1} P u): (I - M^n) u with the operators cached at slot s (Eq. advection_disc).
__global__ void __launch_bounds__(256) k_advect(VesIndex vi, const double* __restrict__ xy,
                                                const double* __restrict__ u,
                                                PointGeom g, const double* __restrict__ tab,
                                                const double* __restrict__ scratch, int s, const int* __restrict__ piv,
                                                double dt, double* __restrict__ xy_out) {
  __shared__ double d[NMAX], u1[NMAX], u2[NMAX], b[2 * NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i < N) {
    d[i] = tab[vi.toff[v] + i];
    u1[i] = u[2 * o + i];
    u2[i] = u[2 * o + N + i];
  }
  __syncthreads();
  if (i < N) b[i] = (g.tx[o + i] * circ_row(d, u1, N, i) + g.ty[o + i] * circ_row(d, u2, N, i)) / g.sa[o + i];
  __syncthreads();
  const double* base = scratch + vi.moff[v];
  const int64_t NN = (int64_t)N * N;
  lu_solve_vec(base + (MatLayout::slot(s) + MatLayout::L) * NN, piv + 4 * o + s * N, N, b);
  const double* T = base + (MatLayout::slot(s) + MatLayout::T) * NN;
  for (int r = i; r < 2 * N; r += blockDim.x) {
    double ts = 0.0;
    for (int k = 0; k < N; ++k) ts = fma(T[(int64_t)r * N + k], b[k], ts);
    const double u = (r < N) ? u1[r] : u2[r - N];
    xy_out[2 * o + r] = xy[2 * o + r] + dt * (u - ts);
  }
}

// X^{n+1} = A^{-1} X*, A = I - dt (I - M*) B* factored in place (Eq. relaxation_disc).
__global__ void __launch_bounds__(256) k_relax_solve(VesIndex vi, const double* __restrict__ xy_star,
                                                     const double* __restrict__ scratch, const int* __restrict__ piv,
                                                     double* __restrict__ xy_out) {
  __shared__ double b[2 * NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) b[r] = xy_star[2 * o + r];
  __syncthreads();
  lu_solve_vec(scratch + vi.moff[v] + MatLayout::A * (int64_t)N * N, piv + 4 * o + 2 * N, 2 * N, b);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) xy_out[2 * o + r] = b[r];
}

// Equal-arclength redistribution (Sec. 4.2): 6x upsampled speed, cumulative trapezoid arclength,
// lower_bound search of k L / N and linear interpolation for alpha~_k, then the trigonometric
// interpolant of X (and of the velocity u, which the tension step reuses) evaluated at alpha~_k.
__global__ void __launch_bounds__(256) k_redistribute(VesIndex vi, const double* __restrict__ xy_in,
                                                      const double* __restrict__ u, const double* __restrict__ tab,
                                                      double* __restrict__ xy_out, double* __restrict__ u_out) {
  __shared__ double val[4][NMAX];
  __shared__ double sp[6 * NMAX];
  __shared__ double l[6 * NMAX + 1];
  __shared__ double cre[4][NMAX / 2 + 1], cim[4][NMAX / 2 + 1];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int Nu = 6 * N;
  const int64_t o = vi.off[v];
  const double* T = tab + vi.toff[v];
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) {
    val[0][i] = xy_in[2 * o + i];
    val[1][i] = xy_in[2 * o + N + i];
    val[2][i] = u[2 * o + i];
    val[3][i] = u[2 * o + N + i];
  }
  __syncthreads();
  const double* K1 = T + 9 * N;
  for (int q = tid; q < Nu; q += blockDim.x) {
    double xp = 0.0, yp = 0.0;
    int m = q;  // (q - 6 j) mod Nu
    for (int j = 0; j < N; ++j) {
      xp = fma(val[0][j], K1[m], xp);
      yp = fma(val[1][j], K1[m], yp);
      m -= 6;
      if (m < 0) m += Nu;
    }
    sp[q] = sqrt(xp * xp + yp * yp);
  }
  __syncthreads();
  const double dal = 2.0 * VS_PI / Nu;
  if (tid == 0) {
    double acc = 0.0;
    l[0] = 0.0;
    for (int q = 0; q < Nu; ++q) {
      acc += 0.5 * dal * (sp[q] + sp[(q + 1 == Nu) ? 0 : q + 1]);
      l[q + 1] = acc;
    }
  }
  // Fourier coefficients c_k = (1/N) sum_j v_j e^{-2 pi i k j / N}, k = 0..N/2, of the 4 fields
  const double* C = T + 15 * N;
  const double* Sn = T + 16 * N;
  const int nk = N / 2 + 1;
  for (int e = tid; e < 4 * nk; e += blockDim.x) {
    const int comp = e / nk, k = e - comp * nk;
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < N; ++j) {
      re = fma(val[comp][j], C[m], re);
      im = fma(-val[comp][j], Sn[m], im);
      m += k;
      if (m >= N) m -= N;
    }
    cre[comp][k] = re / N;
    cim[comp][k] = im / N;
  }
  __syncthreads();
  const double total = l[Nu];
  for (int k = tid; k < N; k += blockDim.x) {
    double alpha = 0.0;
    if (k > 0) {
      const double target = k * total / N;
      int lo = 0, hi = Nu + 1;  // first index with l >= target
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (l[mid] < target) lo = mid + 1; else hi = mid;
      }
      const int m1 = lo, m0 = m1 - 1;
      const double frac = (target - l[m0]) / (l[m1] - l[m0]);
      alpha = dal * m0 + frac * dal;
    }
    double c1, s1;
    sincos(alpha, &s1, &c1);
    double out[4];
#pragma unroll
    for (int comp = 0; comp < 4; ++comp) out[comp] = cre[comp][0];
    double cm = c1, sm = s1;
    for (int mm = 1; mm < N / 2; ++mm) {
#pragma unroll
      for (int comp = 0; comp < 4; ++comp) out[comp] += 2.0 * (cre[comp][mm] * cm - cim[comp][mm] * sm);
      const double cn = cm * c1 - sm * s1;
      sm = sm * c1 + cm * s1;
      cm = cn;
    }
    const double cN = cos((N / 2) * alpha);
#pragma unroll
    for (int comp = 0; comp < 4; ++comp) out[comp] += cre[comp][N / 2] * cN;
    xy_out[2 * o + k] = out[0];
    xy_out[2 * o + N + k] = out[1];
    u_out[2 * o + k] = out[2];
    u_out[2 * o + N + k] = out[3];
  }
}

// sigma = -L^{-1} P (B X + u) at slot s (Eq. tension_disc), with B X = -kappa S X_ssss.
__global__ void __launch_bounds__(256) k_tension(VesIndex vi, const double* __restrict__ bx,
                                                 const double* __restrict__ by, const double* __restrict__ u,
                                                 PointGeom g,
                                                 const double* __restrict__ tab, const double* __restrict__ scratch,
                                                 int s, const int* __restrict__ piv, double kappa,
                                                 double* __restrict__ sigma) {
  __shared__ double d[NMAX], b[2 * NMAX], w[2 * NMAX], rhs[NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i < N) {
    d[i] = tab[vi.toff[v] + i];
    b[i] = bx[o + i];
    b[N + i] = by[o + i];
  }
  __syncthreads();
  const double* base = scratch + vi.moff[v];
  const int64_t NN = (int64_t)N * N;
  const double* S = base + (MatLayout::slot(s) + MatLayout::S) * NN;
  for (int r = i; r < 2 * N; r += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < 2 * N; ++k) acc = fma(S[(int64_t)r * 2 * N + k], b[k], acc);
    w[r] = -kappa * acc + u[2 * o + r];
  }
  __syncthreads();
  if (i < N) rhs[i] = (g.tx[o + i] * circ_row(d, w, N, i) + g.ty[o + i] * circ_row(d, w + N, N, i)) / g.sa[o + i];
  __syncthreads();
  lu_solve_vec(base + (MatLayout::slot(s) + MatLayout::L) * NN, piv + 4 * o + s * N, N, rhs);
  if (i < N) sigma[o + i] = -rhs[i];
}

// Area and length (Green formula / trapezoid of |X_alpha|) and their gradients at z.
struct AL { double A, L; };

__device__ AL area_length_grad(const double* d, const double* zx, const double* zy, int N,
                               double* gAx, double* gAy, double* gLx, double* gLy, double* tmpx,
                               double* tmpy, double* red) {
  const int i = threadIdx.x;
  const bool act = i < N;
  const double dal = 2.0 * VS_PI / N;
  double xa = 0.0, ya = 0.0, s = 1.0;
  if (act) {
    xa = circ_row(d, zx, N, i);
    ya = circ_row(d, zy, N, i);
    s = sqrt(xa * xa + ya * ya);
  }
  const double A = block_sum(act ? dal * 0.5 * (zx[i] * ya - zy[i] * xa) : 0.0, red);
  const double L = block_sum(act ? dal * s : 0.0, red);
  __syncthreads();
  if (act) { tmpx[i] = xa / s; tmpy[i] = ya / s; }
  __syncthreads();
  if (act) {
    gAx[i] = dal * ya;
    gAy[i] = -dal * xa;
    gLx[i] = -dal * circ_row(d, tmpx, N, i);
    gLy[i] = -dal * circ_row(d, tmpy, N, i);
  }
  __syncthreads();
  return AL{A, L};
}

// Block-wide max of one double (all threads get it).
__device__ inline double block_max(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  return m;
}

// Area/length correction (Sec. 4.3): when a relative error exceeds tol, replace X by the
// minimiser of ||X~ - X||^2 subject to A = A_0, L = L_0. The KKT point X~ = X + J(X~)^T lam,
// c(X~) = 0 is reached by the fixed-point iteration z <- X + J(z)^T lam, lam solving
// c(X + J(z)^T lam) = 0 by 2x2 Newton steps. Sets dirty[v] when it fires, clears it otherwise.
__global__ void __launch_bounds__(NMAX) k_correct(VesIndex vi, double* __restrict__ xy,
                                                  const double* __restrict__ A0, const double* __restrict__ L0,
                                                  double tol, const double* __restrict__ tab, int* __restrict__ dirty,
                                                  int* __restrict__ fired, unsigned* err) {
  __shared__ double d[NMAX], X0x[NMAX], X0y[NMAX], zx[NMAX], zy[NMAX], yx[NMAX], yy[NMAX];
  __shared__ double jAx[NMAX], jAy[NMAX], jLx[NMAX], jLy[NMAX];
  __shared__ double hAx[NMAX], hAy[NMAX], hLx[NMAX], hLy[NMAX], t1[NMAX], t2[NMAX], red[NMAX / 32];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const bool act = i < N;
  if (act) {
    d[i] = tab[vi.toff[v] + i];
    X0x[i] = xy[2 * o + i];
    X0y[i] = xy[2 * o + N + i];
    zx[i] = X0x[i];
    zy[i] = X0y[i];
  }
  const int bad = __syncthreads_or(act && !(isfinite(X0x[i]) && isfinite(X0y[i])));
  if (bad) {
    if (i == 0) atomicOr(err, ERR_NONFINITE);
    return;
  }
  const double a0 = A0[v], l0 = L0[v];
  const AL c0 = area_length_grad(d, zx, zy, N, jAx, jAy, jLx, jLy, t1, t2, red);
  if (!(fabs(c0.A - a0) / fabs(a0) > tol || fabs(c0.L - l0) / fabs(l0) > tol)) {
    if (i == 0) dirty[v] = 0;
    return;
  }
  const double xmax = block_max(act ? fmax(fabs(X0x[i]), fabs(X0y[i])) : 0.0, red);
  double la = 0.0, ll = 0.0;
  bool converged = false;
  for (int outer = 0; outer < 60 && !converged; ++outer) {
    // jA, jL hold the constraint gradients at the current iterate z
    for (int inner = 0; inner < 40; ++inner) {
      __syncthreads();
      if (act) {
        yx[i] = X0x[i] + la * jAx[i] + ll * jLx[i];
        yy[i] = X0y[i] + la * jAy[i] + ll * jLy[i];
      }
      __syncthreads();
      const AL cy = area_length_grad(d, yx, yy, N, hAx, hAy, hLx, hLy, t1, t2, red);
      const double FA = cy.A - a0, FL = cy.L - l0;
      const double J11 = block_sum(act ? hAx[i] * jAx[i] + hAy[i] * jAy[i] : 0.0, red);
      const double J12 = block_sum(act ? hAx[i] * jLx[i] + hAy[i] * jLy[i] : 0.0, red);
      const double J21 = block_sum(act ? hLx[i] * jAx[i] + hLy[i] * jAy[i] : 0.0, red);
      const double J22 = block_sum(act ? hLx[i] * jLx[i] + hLy[i] * jLy[i] : 0.0, red);
      if (fabs(FA) <= 1e-15 * fabs(a0) && fabs(FL) <= 1e-15 * fabs(l0)) break;
      const double det = J11 * J22 - J12 * J21;
      const double nrm = J11 * J11 + J12 * J12 + J21 * J21 + J22 * J22;
      double dA, dL;
      if (fabs(det) > 1e-12 * nrm) {
        dA = (J22 * FA - J12 * FL) / det;
        dL = (-J21 * FA + J11 * FL) / det;
      } else {  // rank-one J (a circle): minimum-norm step
        dA = (J11 * FA + J21 * FL) / nrm;
        dL = (J12 * FA + J22 * FL) / nrm;
      }
      la -= dA;
      ll -= dL;
    }
    __syncthreads();
    double dz = 0.0;
    if (act) {
      const double nx = X0x[i] + la * jAx[i] + ll * jLx[i];
      const double ny = X0y[i] + la * jAy[i] + ll * jLy[i];
      dz = fmax(fabs(nx - zx[i]), fabs(ny - zy[i]));
      yx[i] = nx;
      yy[i] = ny;
    }
    const double step = block_max(dz, red);
    if (act) { zx[i] = yx[i]; zy[i] = yy[i]; }
    __syncthreads();
    converged = step <= 1e-15 * xmax;
    if (!converged) area_length_grad(d, zx, zy, N, jAx, jAy, jLx, jLy, t1, t2, red);
  }
  if (!converged && i == 0) atomicOr(err, ERR_CORRECTION);
  if (act) {
    xy[2 * o + i] = zx[i];
    xy[2 * o + N + i] = zy[i];
  }
  if (i == 0) {
    dirty[v] = 1;
    atomicAdd(fired, 1);
  }
}

}  // namespace vs
