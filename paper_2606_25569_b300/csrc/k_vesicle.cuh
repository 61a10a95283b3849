// Per-vesicle step kernels: advection, relaxation solve, redistribution, tension, correction
// (Eqs. advection_disc, relaxation_disc, tension_disc; Sec. 4.2, 4.3). One CTA per vesicle.
#pragma once
#include "common.cuh"
#include "dfloat.cuh"
#include "k_dense.cuh"

namespace vs {

struct PointGeom {
  const double* sa;
  const double* tx;
  const double* ty;
};

// X* = X^n + dt (u - T L^{-1} P u): (I - M^n) u with the operators cached at slot s (Eq. advection_disc);
// with `active`, only the vesicles flagged there.
__global__ void __launch_bounds__(256) k_advect(VesIndex vi, const double* __restrict__ xy,
                                                const double* __restrict__ u,
                                                PointGeom g, const double* __restrict__ tab,
                                                const double* __restrict__ scratch, int s, const int* __restrict__ piv,
                                                double dt, double* __restrict__ xy_out,
                                                const int* __restrict__ active = nullptr) {
  __shared__ double d[NMAX], u1[NMAX], u2[NMAX], b[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
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
                                                     double* __restrict__ xy_out, const int* __restrict__ active) {
  __shared__ double b[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
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
  // sums of products run in double-float (FP64 is 1/64 of the FP32 rate on this part); the positions
  // enter relative to point 0 and the mean is restored on output
  __shared__ float2 val[4][NMAX];
  __shared__ float2 k1[6 * NMAX], cs[NMAX], sn[NMAX];
  __shared__ double sp[6 * NMAX];
  __shared__ double l[6 * NMAX + 1];
  __shared__ float2 cre[4][NMAX / 2 + 1], cim[4][NMAX / 2 + 1];
  __shared__ double base[2];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int Nu = 6 * N;
  const int64_t o = vi.off[v];
  const double* T = tab + vi.toff[v];
  const int tid = threadIdx.x;
  if (tid < 2) base[tid] = xy_in[2 * o + tid * N];
  __syncthreads();
  for (int i = tid; i < N; i += blockDim.x) {
    val[0][i] = df_of(xy_in[2 * o + i] - base[0]);
    val[1][i] = df_of(xy_in[2 * o + N + i] - base[1]);
    val[2][i] = df_of(u[2 * o + i]);
    val[3][i] = df_of(u[2 * o + N + i]);
    cs[i] = df_of(T[15 * N + i]);
    sn[i] = df_of(T[16 * N + i]);
  }
  for (int q = tid; q < Nu; q += blockDim.x) k1[q] = df_of(T[9 * N + q]);
  __syncthreads();
  // speed |X_alpha| on the 6x finer grid from the interpolation kernel's derivative
  for (int q = tid; q < Nu; q += blockDim.x) {
    float2 xp = make_float2(0.f, 0.f), yp = xp;
    int m = q;  // (q - 6 j) mod Nu
    for (int j0 = 0; j0 < N; j0 += DF_CHUNK) {
      Dot2 ax, ay;
      const int j1 = min(j0 + DF_CHUNK, N);
      for (int j = j0; j < j1; ++j) {
        ax.add(val[0][j], k1[m]);
        ay.add(val[1][j], k1[m]);
        m -= 6;
        if (m < 0) m += Nu;
      }
      xp = df_add(xp, ax.value());
      yp = df_add(yp, ay.value());
    }
    const double x = df_val(xp), y = df_val(yp);
    sp[q] = sqrt(x * x + y * y);
  }
  __syncthreads();
  // cumulative trapezoid of the speed: warp 0, each lane a contiguous segment, then a shuffle scan
  const double dal = 2.0 * VS_PI / Nu;
  if (tid < 32) {
    const int seg = (Nu + 31) / 32, q0 = tid * seg, q1 = min(q0 + seg, Nu);
    double acc = 0.0;
    for (int q = q0; q < q1; ++q) acc += 0.5 * dal * (sp[q] + sp[(q + 1 == Nu) ? 0 : q + 1]);
    double incl = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, incl, off);
      if (tid >= off) incl += t;
    }
    double run = incl - acc;
    if (tid == 0) l[0] = 0.0;
    for (int q = q0; q < q1; ++q) {
      run += 0.5 * dal * (sp[q] + sp[(q + 1 == Nu) ? 0 : q + 1]);
      l[q + 1] = run;
    }
  }
  // Fourier coefficients c_k = (1/N) sum_j v_j e^{-2 pi i k j / N}, k = 0..N/2, of the 4 fields
  const int nk = N / 2 + 1;
  const float2 invN = df_of(1.0 / N);
  for (int e = tid; e < 4 * nk; e += blockDim.x) {
    const int comp = e / nk, k = e - comp * nk;
    float2 re = make_float2(0.f, 0.f), im = re;
    int m = 0;
    for (int j0 = 0; j0 < N; j0 += DF_CHUNK) {
      Dot2 ar, ai;
      const int j1 = min(j0 + DF_CHUNK, N);
      for (int j = j0; j < j1; ++j) {
        ar.add(val[comp][j], cs[m]);
        ai.add(val[comp][j], sn[m]);
        m += k;
        if (m >= N) m -= N;
      }
      re = df_add(re, ar.value());
      im = df_add(im, ai.value());
    }
    cre[comp][k] = df_mul(re, invN);
    cim[comp][k] = df_mul(make_float2(-im.x, -im.y), invN);
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
    double c1d, s1d;
    sincos(alpha, &s1d, &c1d);
    const float2 c1 = df_of(c1d), s1 = df_of(s1d);
    // trigonometric interpolant: c_0 + 2 sum_{m < N/2} Re(c_m e^{i m alpha}) + c_{N/2} cos(N alpha / 2)
    float2 out[4];
    Dot2 acc[4];
#pragma unroll
    for (int comp = 0; comp < 4; ++comp) out[comp] = cre[comp][0];
    float2 cm = c1, sm = s1;
    for (int mm = 1; mm < N / 2; ++mm) {
#pragma unroll
      for (int comp = 0; comp < 4; ++comp) {
        acc[comp].add(cre[comp][mm], cm);
        acc[comp].add(make_float2(-cim[comp][mm].x, -cim[comp][mm].y), sm);
      }
      const float2 cn = df_add(df_mul(cm, c1), make_float2(-df_mul(sm, s1).x, -df_mul(sm, s1).y));
      sm = df_add(df_mul(sm, c1), df_mul(cm, s1));
      cm = cn;
      if ((mm & (DF_CHUNK - 1)) == 0) {
#pragma unroll
        for (int comp = 0; comp < 4; ++comp) {
          const float2 a = acc[comp].value();
          out[comp] = df_add(out[comp], make_float2(2.f * a.x, 2.f * a.y));
          acc[comp] = Dot2();
        }
      }
    }
    const double cN = cos((N / 2) * alpha);
    double res[4];
#pragma unroll
    for (int comp = 0; comp < 4; ++comp) {
      const float2 a = acc[comp].value();
      out[comp] = df_add(out[comp], make_float2(2.f * a.x, 2.f * a.y));
      res[comp] = df_val(out[comp]) + df_val(cre[comp][N / 2]) * cN;
    }
    xy_out[2 * o + k] = res[0] + base[0];
    xy_out[2 * o + N + k] = res[1] + base[1];
    u_out[2 * o + k] = res[2];
    u_out[2 * o + N + k] = res[3];
  }
}

// sigma = -L^{-1} P (B X + u) at slot s (Eq. tension_disc), with B X = -kappa S X_ssss; with `active`, only
// the vesicles flagged there.
__global__ void __launch_bounds__(256) k_tension(VesIndex vi, const double* __restrict__ bx,
                                                 const double* __restrict__ by, const double* __restrict__ u,
                                                 PointGeom g,
                                                 const double* __restrict__ tab, const double* __restrict__ scratch,
                                                 int s, const int* __restrict__ piv, double kappa,
                                                 double* __restrict__ sigma, const int* __restrict__ active = nullptr) {
  __shared__ double d[NMAX], b[2 * NMAX], w[2 * NMAX], rhs[NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
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

// Area/length correction (Sec. 4.3) as the exact constrained minimiser of ||X~ - X||^2 subject to
// A(X~) = A_0, L(X~) = L_0, found by Newton's method on its KKT system
//   [ I - lam_A H_A - lam_L H_L   -J^T ] [dz  ]     [ z - X - J^T lam ]
//   [ J                            0   ] [dlam] = - [ c(z)            ]
// with the discrete A = (2 pi/N) sum 1/2 (x y' - y x'), L = (2 pi/N) sum |X'|, X' = D X, their
// gradients J = (grad A, grad L) and exact Hessians H_A = (2 pi/N)[[0, D], [D^T, 0]],
// H_L = (2 pi/N) blockdiag(D, D)^T Q blockdiag(D, D), Q = (I - t t^T)/|X'| per point. Coordinates are
// taken relative to the mean point. Per vesicle state (6 N + 16 doubles at 6 off + 16 v): X0 (2N),
// z (2N), rhs (2N + 2), then lam_A, lam_L, mean_x, mean_y, size, converged. The (2N+2)^2 system
// lives in the vesicle's matrix scratch from MatLayout::B (free at this point of the step).

__device__ __forceinline__ double* corr_state(double* corr, const VesIndex& vi, int v) {
  return corr + 6 * vi.off[v] + 16 * (int64_t)v;
}

// Trigger test (relative error of A or L above tol) and Newton start z = X, lam = 0.
__global__ void __launch_bounds__(NMAX) k_corr_init(VesIndex vi, const double* __restrict__ xy,
                                                    const double* __restrict__ A0, const double* __restrict__ L0,
                                                    double tol, const double* __restrict__ tab,
                                                    double* __restrict__ corr, int* __restrict__ active,
                                                    int* __restrict__ dirty, unsigned* err) {
  __shared__ double d[NMAX], xs[NMAX], ys[NMAX], red[NMAX / 32];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const bool act = i < N;
  const double px = act ? xy[2 * o + i] : 0.0, py = act ? xy[2 * o + N + i] : 0.0;
  if (__syncthreads_or(act && !(isfinite(px) && isfinite(py)))) {
    if (i == 0) { atomicOr(err, ERR_NONFINITE); active[v] = 0; dirty[v] = 0; }
    return;
  }
  const double mx = block_sum(px, red) / N, my = block_sum(py, red) / N;
  if (act) {
    d[i] = tab[vi.toff[v] + i];
    xs[i] = px - mx;
    ys[i] = py - my;
  }
  __syncthreads();
  double xa = 0.0, ya = 0.0;
  if (act) {
    xa = circ_row(d, xs, N, i);
    ya = circ_row(d, ys, N, i);
  }
  const double dal = 2.0 * VS_PI / N;
  const double A = block_sum(act ? dal * 0.5 * (xs[i] * ya - ys[i] * xa) : 0.0, red);
  const double L = block_sum(act ? dal * sqrt(xa * xa + ya * ya) : 0.0, red);
  double size = act ? fmax(fabs(xs[i]), fabs(ys[i])) : 0.0;
  for (int off = 16; off > 0; off >>= 1) size = fmax(size, __shfl_xor_sync(0xffffffffu, size, off));
  __syncthreads();
  if ((i & 31) == 0) red[i >> 5] = size;
  __syncthreads();
  size = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) size = fmax(size, red[w]);
  const bool fire = fabs(A - A0[v]) / fabs(A0[v]) > tol || fabs(L - L0[v]) / fabs(L0[v]) > tol;
  double* st = corr_state(corr, vi, v);
  if (fire && act) {
    st[i] = xs[i];
    st[N + i] = ys[i];
    st[2 * N + i] = xs[i];
    st[3 * N + i] = ys[i];
  }
  if (i == 0) {
    active[v] = fire ? 1 : 0;
    dirty[v] = fire ? 1 : 0;
    double* sc = st + 6 * N + 2;
    sc[0] = 0.0; sc[1] = 0.0; sc[2] = mx; sc[3] = my; sc[4] = size; sc[5] = 0.0;
  }
}

// Assemble the KKT matrix K (n x n, n = 2N + 2, in the B block of the scratch) and the right-hand side
// at the current iterate of vesicle v.
__device__ void corr_build(int v, VesIndex vi, const double* __restrict__ tab, const double* __restrict__ A0,
                           const double* __restrict__ L0, double* __restrict__ corr, double* __restrict__ scratch) {
  __shared__ double d[NMAX], zx[NMAX], zy[NMAX], tx[NMAX], ty[NMAX], qxx[NMAX], qxy[NMAX], qyy[NMAX];
  __shared__ double gA[2 * NMAX], gL[2 * NMAX], red[8];
  const int N = vi.N[v];
  const int n = 2 * N + 2;
  const int tid = threadIdx.x;
  double* st = corr_state(corr, vi, v);
  const double la = st[6 * N + 2], ll = st[6 * N + 3];
  for (int i = tid; i < N; i += blockDim.x) {
    d[i] = tab[vi.toff[v] + i];
    zx[i] = st[2 * N + i];
    zy[i] = st[3 * N + i];
  }
  __syncthreads();
  const double dal = 2.0 * VS_PI / N;
  double pa = 0.0, pl = 0.0;
  for (int i = tid; i < N; i += blockDim.x) {
    const double xa = circ_row(d, zx, N, i), ya = circ_row(d, zy, N, i);
    const double sp = sqrt(xa * xa + ya * ya);
    tx[i] = xa / sp;
    ty[i] = ya / sp;
    qxx[i] = ty[i] * ty[i] / sp;
    qxy[i] = -tx[i] * ty[i] / sp;
    qyy[i] = tx[i] * tx[i] / sp;
    gA[i] = dal * ya;
    gA[N + i] = -dal * xa;
    pa += dal * 0.5 * (zx[i] * ya - zy[i] * xa);
    pl += dal * sp;
  }
  const double Acur = block_sum(pa, red), Lcur = block_sum(pl, red);
  __syncthreads();
  for (int i = tid; i < N; i += blockDim.x) {
    gL[i] = -dal * circ_row(d, tx, N, i);
    gL[N + i] = -dal * circ_row(d, ty, N, i);
  }
  __syncthreads();
  double* K = scratch + vi.moff[v] + MatLayout::B * (int64_t)N * N;
  for (int e = tid; e < 2 * N * 2 * N; e += blockDim.x) {
    const int a = e / (2 * N), b = e - a * (2 * N);
    const int p = a / N, i = a - p * N, q = b / N, j = b - q * N;
    double hl = 0.0;
    for (int k = 0; k < N; ++k) {
      int ki = k - i, kj = k - j;
      ki += (ki < 0) ? N : 0;
      kj += (kj < 0) ? N : 0;
      const double qq = (p == 0) ? ((q == 0) ? qxx[k] : qxy[k]) : ((q == 0) ? qxy[k] : qyy[k]);
      hl = fma(d[ki] * d[kj], qq, hl);
    }
    double ha = 0.0;
    if (p == 0 && q == 1) { int m = i - j; m += (m < 0) ? N : 0; ha = d[m]; }
    if (p == 1 && q == 0) { int m = j - i; m += (m < 0) ? N : 0; ha = d[m]; }
    K[(int64_t)a * n + b] = ((a == b) ? 1.0 : 0.0) - la * dal * ha - ll * dal * hl;
  }
  for (int a = tid; a < 2 * N; a += blockDim.x) {
    K[(int64_t)a * n + 2 * N] = -gA[a];
    K[(int64_t)a * n + 2 * N + 1] = -gL[a];
    K[(int64_t)(2 * N) * n + a] = gA[a];
    K[(int64_t)(2 * N + 1) * n + a] = gL[a];
    const double z = (a < N) ? zx[a] : zy[a - N];
    st[4 * N + a] = -(z - st[a] - la * gA[a] - ll * gL[a]);
  }
  if (tid == 0) {
    K[(int64_t)(2 * N) * n + 2 * N] = 0.0;
    K[(int64_t)(2 * N) * n + 2 * N + 1] = 0.0;
    K[(int64_t)(2 * N + 1) * n + 2 * N] = 0.0;
    K[(int64_t)(2 * N + 1) * n + 2 * N + 1] = 0.0;
    st[6 * N] = -(Acur - A0[v]);
    st[6 * N + 1] = -(Lcur - L0[v]);
  }
}

// Solve the KKT system factored in LU (pivots p), update (z, lam), retire the vesicle once converged.
__device__ void corr_update(int v, VesIndex vi, const double* LU, const int* p, double* __restrict__ corr,
                            int* __restrict__ active) {
  __shared__ double b[2 * NMAX + 8], red[8];
  const int N = vi.N[v];
  const int n = 2 * N + 2;
  double* st = corr_state(corr, vi, v);
  for (int a = threadIdx.x; a < n; a += blockDim.x) b[a] = st[4 * N + a];
  __syncthreads();
  lu_solve_vec(LU, p, n, b);
  double dm = 0.0;
  for (int a = threadIdx.x; a < 2 * N; a += blockDim.x) {
    st[2 * N + a] += b[a];
    dm = fmax(dm, fabs(b[a]));
  }
  for (int off = 16; off > 0; off >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    st[6 * N + 2] += b[2 * N];
    st[6 * N + 3] += b[2 * N + 1];
    if (m <= 1e-14 * st[6 * N + 6]) {
      st[6 * N + 7] = 1.0;
      active[v] = 0;
    }
  }
}

// Newton iterations of the correction with an FP32 Jacobian (2N <= 16 RA): per step the FP64 residual
// (z - X - J^T lam, c(z)) as in corr_build, the 2N x 2N block M = I - lam_A H_A - lam_L H_L assembled in
// FP32 in dynamic shared memory and inverted in registers (gj_invert_np, else gj_invert), and the KKT system
//   [M  -G; G^T  0] [dz; dlam] = [r1; r2],  G = (grad A, grad L)
// solved through its 2 x 2 Schur complement: y = M^{-1} r1, Y = M^{-1} G, (G^T Y) dlam = r2 - G^T y,
// dz = y + Y dlam. The FP32 Jacobian makes the iteration converge linearly (factor about 1e-6) to the
// same KKT point that the FP64 residual defines, and so does keeping M's inverse from one step to the
// next (chord steps) while the updates keep shrinking; the same stopping test as corr_update. 256 threads.
template <int RA>
__global__ void __launch_bounds__(256) k_corr_newton32(VesIndex vi, const double* __restrict__ tab,
                                                       const double* __restrict__ A0, const double* __restrict__ L0,
                                                       double* __restrict__ corr, int* __restrict__ active,
                                                       const int* __restrict__ dirty, int iters,
                                                       double* __restrict__ xy, int* __restrict__ fired, unsigned* err) {
  extern __shared__ __align__(16) float Mg[];  // (2N)^2
  __shared__ double d[NMAX], zx[NMAX], zy[NMAX], gA[2 * NMAX], gL[2 * NMAX], r1[2 * NMAX], red[8];
  __shared__ float dq[NMAX], qxx[NMAX], qxy[NMAX], qyy[NMAX];
  __shared__ float yv[3][2 * NMAX];
  __shared__ double sol[3];
  const int v = vi.vid(blockIdx.x);
  if (!dirty[v]) return;
  const int N = vi.N[v];
  const int n2 = 2 * N;
  const int tid = threadIdx.x;
  double* st = corr_state(corr, vi, v);
  const double dal = 2.0 * VS_PI / N;
  for (int i = tid; i < N; i += blockDim.x) {
    d[i] = tab[vi.toff[v] + i];
    dq[i] = (float)d[i];
  }
  // the inverse of M is formed on the first step (M = I at lam = 0), re-formed on the second and kept
  // while each update shrinks by 10x or more (a chord iteration on the Jacobian of the second step)
  __shared__ int reinv;
  __shared__ double mprev;
  if (tid == 0) { reinv = 1; mprev = 1e300; }
  for (int it = 0; it < iters; ++it) {
    __syncthreads();
    if (!active[v]) break;  // uniform: written by thread 0 of this CTA before the barrier
    const double la = st[6 * N + 2], ll = st[6 * N + 3];
    for (int i = tid; i < N; i += blockDim.x) {
      zx[i] = st[2 * N + i];
      zy[i] = st[3 * N + i];
    }
    __syncthreads();
    // geometry of z and the FP64 residual (same formulas as corr_build)
    double pa = 0.0, pl = 0.0;
    __shared__ double txs[NMAX], tys[NMAX];
    for (int i = tid; i < N; i += blockDim.x) {
      const double xa = circ_row(d, zx, N, i), ya = circ_row(d, zy, N, i);
      const double sp = sqrt(xa * xa + ya * ya);
      txs[i] = xa / sp;
      tys[i] = ya / sp;
      qxx[i] = (float)(tys[i] * tys[i] / sp);
      qxy[i] = (float)(-txs[i] * tys[i] / sp);
      qyy[i] = (float)(txs[i] * txs[i] / sp);
      gA[i] = dal * ya;
      gA[N + i] = -dal * xa;
      pa += dal * 0.5 * (zx[i] * ya - zy[i] * xa);
      pl += dal * sp;
    }
    const double Acur = block_sum(pa, red), Lcur = block_sum(pl, red);
    __syncthreads();
    for (int i = tid; i < N; i += blockDim.x) {
      gL[i] = -dal * circ_row(d, txs, N, i);
      gL[N + i] = -dal * circ_row(d, tys, N, i);
    }
    __syncthreads();
    for (int a = tid; a < n2; a += blockDim.x) {
      const double z = (a < N) ? zx[a] : zy[a - N];
      r1[a] = -(z - st[a] - la * gA[a] - ll * gL[a]);
    }
    // M = I - la dal H_A - ll dal H_L in FP32
    const float fa = (float)(la * dal), fl = (float)(ll * dal);
    if (reinv && it == 0 && la == 0.0 && ll == 0.0) {
      for (int e = tid; e < n2 * n2; e += blockDim.x) Mg[e] = (e / n2 == e % n2) ? 1.f : 0.f;
    } else if (reinv) {
      for (int e = tid; e < n2 * n2; e += blockDim.x) {
        const int a = e / n2, b = e - a * n2;
        const int p = a / N, i = a - p * N, q = b / N, j = b - q * N;
        const float* qq = (p == 0) ? ((q == 0) ? qxx : qxy) : ((q == 0) ? qxy : qyy);
        float hl = 0.f;
        int ki = N - i, kj = N - j;  // (k - i) mod N at k = 0
        if (ki == N) ki = 0;
        if (kj == N) kj = 0;
        for (int k = 0; k < N; ++k) {
          hl = fmaf(dq[ki] * dq[kj], qq[k], hl);
          if (++ki == N) ki = 0;
          if (++kj == N) kj = 0;
        }
        float ha = 0.f;
        if (p == 0 && q == 1) { int m = i - j; m += (m < 0) ? N : 0; ha = dq[m]; }
        if (p == 1 && q == 0) { int m = j - i; m += (m < 0) ? N : 0; ha = dq[m]; }
        Mg[e] = ((a == b) ? 1.f : 0.f) - fa * ha - fl * hl;
      }
      __syncthreads();
      if (!gj_invert_np<RA, RA, 16>(Mg, Mg, n2)) gj_invert<RA, RA, 16>(Mg, Mg, n2, err);
    }
    __syncthreads();
    // y = M^{-1} r1, Y = M^{-1} (gA, gL): warp per row
    {
      const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
      for (int a = wid; a < n2; a += nw) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int b = lane; b < n2; b += 32) {
          const float m = Mg[a * n2 + b];
          s0 = fmaf(m, (float)r1[b], s0);
          s1 = fmaf(m, (float)gA[b], s1);
          s2 = fmaf(m, (float)gL[b], s2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          s0 += __shfl_xor_sync(0xffffffffu, s0, o);
          s1 += __shfl_xor_sync(0xffffffffu, s1, o);
          s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) { yv[0][a] = s0; yv[1][a] = s1; yv[2][a] = s2; }
      }
    }
    __syncthreads();
    // 2 x 2 Schur system (G^T Y) dlam = r2 - G^T y in FP64 (warp 0)
    if (tid < 32) {
      double gy[2] = {0.0, 0.0}, S[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
      for (int a = tid; a < n2; a += 32) {
        const double y0 = yv[0][a], ya = yv[1][a], yl = yv[2][a];
        gy[0] += gA[a] * y0;
        gy[1] += gL[a] * y0;
        S[0][0] += gA[a] * ya;
        S[0][1] += gA[a] * yl;
        S[1][0] += gL[a] * ya;
        S[1][1] += gL[a] * yl;
      }
      gy[0] = warp_sum(gy[0]);
      gy[1] = warp_sum(gy[1]);
      S[0][0] = warp_sum(S[0][0]);
      S[0][1] = warp_sum(S[0][1]);
      S[1][0] = warp_sum(S[1][0]);
      S[1][1] = warp_sum(S[1][1]);
      if (tid == 0) {
        const double b0 = -(Acur - A0[v]) - gy[0], b1 = -(Lcur - L0[v]) - gy[1];
        const double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
        const double idet = (det != 0.0) ? 1.0 / det : 0.0;
        sol[0] = (b0 * S[1][1] - b1 * S[0][1]) * idet;
        sol[1] = (S[0][0] * b1 - S[1][0] * b0) * idet;
        if (det == 0.0) atomicOr(err, ERR_PIVOT);
      }
    }
    __syncthreads();
    const double dla = sol[0], dll = sol[1];
    double dm = 0.0;
    for (int a = tid; a < n2; a += blockDim.x) {
      const double dz = (double)yv[0][a] + (double)yv[1][a] * dla + (double)yv[2][a] * dll;
      st[2 * N + a] += dz;
      dm = fmax(dm, fabs(dz));
    }
    for (int off = 16; off > 0; off >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, off));
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dm;
    __syncthreads();
    if (tid == 0) {
      double m = red[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
      st[6 * N + 2] += dla;
      st[6 * N + 3] += dll;
      if (m <= 1e-14 * st[6 * N + 6]) {
        st[6 * N + 7] = 1.0;
        active[v] = 0;
      }
      reinv = (it == 0) || !(m <= 0.1 * mprev);
      mprev = m;
    }
  }
  __syncthreads();
  const int64_t o = vi.off[v];
  for (int i = tid; i < N; i += blockDim.x) {
    xy[2 * o + i] = st[2 * N + i] + st[6 * N + 4];
    xy[2 * o + N + i] = st[3 * N + i] + st[6 * N + 5];
  }
  if (tid == 0) {
    atomicAdd(fired, 1);
    if (st[6 * N + 7] == 0.0) atomicOr(err, ERR_CORRECTION);
  }
}

// Newton iterations of the correction for every vesicle flagged by k_corr_init (dirty), at most `iters`
// steps: assemble K, factor it (in dynamic shared memory when SMEM, else in place), solve, update; then
// write the corrected points back (plus the mean) and flag vesicles that did not converge. One CTA of
// 256 threads per vesicle.
template <bool SMEM>
__global__ void __launch_bounds__(256) k_corr_newton(VesIndex vi, const double* __restrict__ tab,
                                                     const double* __restrict__ A0, const double* __restrict__ L0,
                                                     double* __restrict__ corr, double* __restrict__ scratch,
                                                     int* __restrict__ cpiv, int* __restrict__ active,
                                                     const int* __restrict__ dirty, int iters,
                                                     double* __restrict__ xy, int* __restrict__ fired, unsigned* err) {
  extern __shared__ unsigned char corr_raw[];
  const int v = vi.vid(blockIdx.x);
  if (!dirty[v]) return;
  const int N = vi.N[v];
  const int n = 2 * N + 2;
  double* K = scratch + vi.moff[v] + MatLayout::B * (int64_t)N * N;
  double* F = SMEM ? reinterpret_cast<double*>(corr_raw) : K;
  int* p = cpiv + 2 * vi.off[v] + 2 * v;
  for (int it = 0; it < iters; ++it) {
    __syncthreads();
    if (!active[v]) break;  // uniform: written by thread 0 of this CTA before the barrier
    corr_build(v, vi, tab, A0, L0, corr, scratch);
    __syncthreads();
    if (SMEM)
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) F[e] = K[e];
    __syncthreads();
    lu_factor<LuGeo>(F, n, p, err);
    __syncthreads();
    corr_update(v, vi, F, p, corr, active);
  }
  __syncthreads();
  const int64_t o = vi.off[v];
  const double* st = corr + 6 * o + 16 * (int64_t)v;
  const int i = threadIdx.x;
  if (i < N) {
    xy[2 * o + i] = st[2 * N + i] + st[6 * N + 4];
    xy[2 * o + N + i] = st[3 * N + i] + st[6 * N + 5];
  }
  if (i == 0) {
    atomicAdd(fired, 1);
    if (st[6 * N + 7] == 0.0) atomicOr(err, ERR_CORRECTION);
  }
}

// New positions for every vesicle: xy <- xy_new, and dirty[v] = 1 where any coordinate of v changed
// (bitwise), so the operators cached for unchanged vesicles stay valid. One CTA of NMAX threads per vesicle.
__global__ void __launch_bounds__(NMAX) k_state_update(VesIndex vi, const double* __restrict__ xy_new,
                                                       double* __restrict__ xy, int* __restrict__ dirty) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  bool changed = false;
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
    const double a = xy_new[2 * o + r];
    changed |= __double_as_longlong(a) != __double_as_longlong(xy[2 * o + r]);
    xy[2 * o + r] = a;
  }
  if (__syncthreads_or(changed) && threadIdx.x == 0) dirty[v] = 1;
}

}  // namespace vs
