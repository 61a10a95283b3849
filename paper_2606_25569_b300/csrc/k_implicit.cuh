// Fully implicit step (Sec. 2.2.3, Eq. time_step_sc1): the coupled system of all vesicles, solved by
// flexible GMRES with a block-diagonal preconditioner (the paper's solver: preconditioned GMRES).
//
// Unknowns per vesicle: z = [x(N), y(N), sigma(N)] at 3 off (the "3-block" layout). With every operator at
// X^n, the density f = -kappa D_s^4 X + D_s(sigma X_s) is linear in z, the velocity is
// U = S f + (far field of f from the other vesicles) (+ near-field correction), and the equations are
//     X - dt U = X^n + dt u_inf(X^n),        P U = -P u_inf(X^n).
// The preconditioner is the same system without the other vesicles, solved exactly per vesicle: with
// t = L^{-1} r_sigma,  X = A^{-1} (r_X + dt T t),  sigma = t - W X,  where A = I - dt (I - T L^{-1} P) B and
// W = L^{-1} P B are the relaxation's matrices (Eq. relaxation_disc) formed at X^n.
//
// Kernels (one CTA per vesicle unless stated):
//   k_imp_rhs       b = [X^n + dt u_inf; -P u_inf]
//   k_imp_pack      z0 = [X^n; sigma^n]
//   k_imp_density   f of a vector p into the far field's source buffers (f, g64, src.zw, gsum), u = 0
//   k_imp_apply     q = [p_X - dt (S f + u); P (S f + u)] (u: the far field + near field of f)
//   k_imp_precond   the block-diagonal inverse above from the FP64 LU factors (FP64 operators), or
//   k_imp_precond32 from the FP32 explicit inverses of the mixed-precision path (an approximate inverse)
//   k_imp_unpack    X^{n+1} and sigma^{n+1} (sigma into the first component of a velocity-shaped buffer,
//                   which the redistribution carries to the new parameters)
//   k_gm_*          GMRES vector kernels over n = 3P doubles (grid-stride; dot products per CTA then a
//                   fixed-order reduction, so every result is deterministic)
#pragma once
#include "common.cuh"
#include "k_dense.cuh"
#include "k_geometry.cuh"
#include "k_mp.cuh"
#include "k_vesicle.cuh"

namespace vs {

// D_s v at point i: (1 / |X_alpha|_i) (D_alpha v)_i
__device__ __forceinline__ double imp_ds(const double* d, const double* v, int N, int i, double isa) {
  return circ_row(d, v, N, i) * isa;
}

__global__ void __launch_bounds__(NMAX) k_imp_rhs(VesIndex vi, const double* __restrict__ xy, PointGeom g,
                                                  const double* __restrict__ tab, FlowDev flow, double dt,
                                                  double* __restrict__ b) {
  __shared__ double d[NMAX], ux[NMAX], uy[NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i < N) {
    d[i] = tab[vi.toff[v] + i];
    const double2 u = background_flow(flow, xy[2 * o + i], xy[2 * o + N + i]);
    ux[i] = u.x;
    uy[i] = u.y;
  }
  __syncthreads();
  if (i >= N) return;
  const double isa = 1.0 / g.sa[o + i];
  b[3 * o + i] = xy[2 * o + i] + dt * ux[i];
  b[3 * o + N + i] = xy[2 * o + N + i] + dt * uy[i];
  b[3 * o + 2 * N + i] = -(g.tx[o + i] * imp_ds(d, ux, N, i, isa) + g.ty[o + i] * imp_ds(d, uy, N, i, isa));
}

__global__ void __launch_bounds__(NMAX) k_imp_pack(VesIndex vi, const double* __restrict__ xy,
                                                   const double* __restrict__ sigma, double* __restrict__ z) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i >= N) return;
  z[3 * o + i] = xy[2 * o + i];
  z[3 * o + N + i] = xy[2 * o + N + i];
  z[3 * o + 2 * N + i] = sigma[o + i];
}

// f = -kappa D_s^4 p_X + D_s(p_sigma X_s) with the geometry of X^n; the far field's source buffers get the
// density (the point positions in src.xy and the centres stay those of X^n), the velocity accumulator 0.
__global__ void __launch_bounds__(NMAX) k_imp_density(VesIndex vi, const double* __restrict__ p, PointGeom g,
                                                      const double* __restrict__ tab, double kappa, double mu,
                                                      double* __restrict__ f, double* __restrict__ g64,
                                                      float4* __restrict__ src, float2* __restrict__ gsum,
                                                      double* __restrict__ u) {
  __shared__ double d[NMAX], wx[NMAX], wy[NMAX], red[NMAX / 32];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const bool act = i < N;
  const double isa = act ? 1.0 / g.sa[o + i] : 0.0;
  const double tx = act ? g.tx[o + i] : 0.0, ty = act ? g.ty[o + i] : 0.0;
  if (act) {
    d[i] = tab[vi.toff[v] + i];
    wx[i] = p[3 * o + i];
    wy[i] = p[3 * o + N + i];
  }
  double bx = 0.0, by = 0.0;
  for (int r = 0; r < 4; ++r) {
    __syncthreads();
    if (act) {
      bx = imp_ds(d, wx, N, i, isa);
      by = imp_ds(d, wy, N, i, isa);
    }
    __syncthreads();
    if (act) { wx[i] = bx; wy[i] = by; }
  }
  __syncthreads();
  const double sg = act ? p[3 * o + 2 * N + i] : 0.0;
  if (act) { wx[i] = sg * tx; wy[i] = sg * ty; }
  __syncthreads();
  double fx = 0.0, fy = 0.0;
  if (act) {
    fx = -kappa * bx + imp_ds(d, wx, N, i, isa);
    fy = -kappa * by + imp_ds(d, wy, N, i, isa);
  }
  const double c = act ? (2.0 * VS_PI / N) / (isa * 4.0 * VS_PI * mu) : 0.0;
  const double gsx = block_sum(fx * c, red);
  const double gsy = block_sum(fy * c, red);
  if (act) {
    f[2 * o + i] = fx;
    f[2 * o + N + i] = fy;
    g64[2 * o + i] = fx * c;
    g64[2 * o + N + i] = fy * c;
    const float4 s = src[o + i];
    src[o + i] = make_float4(s.x, s.y, (float)(fx * c), (float)(fy * c));
    u[2 * o + i] = 0.0;
    u[2 * o + N + i] = 0.0;
  }
  if (i == 0) gsum[v] = make_float2((float)gsx, (float)gsy);
}

// q = [p_X - dt w; P w] with w = S f + u (S at slot s).
__global__ void __launch_bounds__(256) k_imp_apply(VesIndex vi, const double* __restrict__ p,
                                                   const double* __restrict__ f, const double* __restrict__ u,
                                                   PointGeom g, const double* __restrict__ tab,
                                                   const double* __restrict__ scratch, int s, double dt,
                                                   double* __restrict__ q) {
  __shared__ double d[NMAX], fs[2 * NMAX], w[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i < N) d[i] = tab[vi.toff[v] + i];
  for (int r = i; r < 2 * N; r += blockDim.x) fs[r] = f[2 * o + r];
  __syncthreads();
  const double* S = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * (int64_t)N * N;
  for (int r = i; r < 2 * N; r += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < 2 * N; ++k) acc = fma(S[(int64_t)r * 2 * N + k], fs[k], acc);
    w[r] = acc + u[2 * o + r];
    q[3 * o + r] = p[3 * o + r] - dt * w[r];
  }
  __syncthreads();
  if (i < N)
    q[3 * o + 2 * N + i] = (g.tx[o + i] * circ_row(d, w, N, i) + g.ty[o + i] * circ_row(d, w + N, N, i)) / g.sa[o + i];
}

// out = the per-vesicle inverse of the self system applied to r (module header). L's LU at slot s, A's LU
// in MatLayout::A (pivots at 2N of the vesicle's pivot block), W = L^{-1} P B in MatLayout::W.
__global__ void __launch_bounds__(256) k_imp_precond(VesIndex vi, const double* __restrict__ r,
                                                     const double* __restrict__ scratch, const int* __restrict__ piv,
                                                     int s, double dt, double* __restrict__ out) {
  __shared__ double t[NMAX], x[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  const int64_t NN = (int64_t)N * N;
  const double* base = scratch + vi.moff[v];
  if (i < N) t[i] = r[3 * o + 2 * N + i];
  __syncthreads();
  lu_solve_vec(base + (MatLayout::slot(s) + MatLayout::L) * NN, piv + 4 * o + s * N, N, t);
  const double* T = base + (MatLayout::slot(s) + MatLayout::T) * NN;
  for (int q = i; q < 2 * N; q += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < N; ++k) acc = fma(T[(int64_t)q * N + k], t[k], acc);
    x[q] = r[3 * o + q] + dt * acc;
  }
  __syncthreads();
  lu_solve_vec(base + MatLayout::A * NN, piv + 4 * o + 2 * N, 2 * N, x);
  const double* W = base + MatLayout::W * NN;
  for (int q = i; q < 2 * N; q += blockDim.x) out[3 * o + q] = x[q];
  if (i < N) {
    double acc = 0.0;
    for (int k = 0; k < 2 * N; ++k) acc = fma(W[(int64_t)i * 2 * N + k], x[k], acc);
    out[3 * o + 2 * N + i] = t[i] - acc;
  }
}

// The same per-vesicle inverse from the FP32 operators of the mixed-precision path (explicit inverses Li32
// of L and Ai32 of A, T32, W32 = Li32 P B32), all arithmetic in FP32: an approximate inverse, which the
// flexible GMRES accepts as it stands (the products with A stay FP64).
template <int THREADS, int COLS>
__global__ void __launch_bounds__(THREADS) k_imp_precond32(VesIndex vi, const double* __restrict__ r,
                                                           const float* __restrict__ scratch32, int s,
                                                           int64_t ainv_sub, double dt, double* __restrict__ out) {
  __shared__ __align__(16) float fs[NMAX], fy[NMAX], fw[NMAX], fr[2 * NMAX], fdx[2 * NMAX];
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int64_t NN = (int64_t)N * N;
  const MpMats m = mp_mats(vi, scratch32, v, s);
  const float* base32 = scratch32 + vi.moff[v];
  for (int i = threadIdx.x; i < N; i += blockDim.x) fs[i] = (float)r[3 * o + 2 * N + i];
  for (int q = threadIdx.x; q < 2 * N; q += blockDim.x) fr[q] = (float)r[3 * o + q];
  __syncthreads();
  matvec32f<COLS>(m.li, N, N, fs, fy, 1.f, false);
  matvec32f<COLS>(m.t32, 2 * N, N, fy, fr, (float)dt, true);
  matvec32f<COLS>(base32 + ainv_sub * NN, 2 * N, 2 * N, fr, fdx, 1.f, false);
  matvec32f<COLS>(base32 + MatLayout::W * NN, N, 2 * N, fdx, fw, 1.f, false);
  for (int q = threadIdx.x; q < 2 * N; q += blockDim.x) out[3 * o + q] = (double)fdx[q];
  for (int i = threadIdx.x; i < N; i += blockDim.x) out[3 * o + 2 * N + i] = (double)fy[i] - (double)fw[i];
}

__global__ void __launch_bounds__(NMAX) k_imp_unpack(VesIndex vi, const double* __restrict__ z,
                                                     double* __restrict__ xy, double* __restrict__ carry) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i >= N) return;
  xy[2 * o + i] = z[3 * o + i];
  xy[2 * o + N + i] = z[3 * o + N + i];
  carry[2 * o + i] = z[3 * o + 2 * N + i];
  carry[2 * o + N + i] = 0.0;
}

// sigma from the first component of the redistributed carrier
__global__ void __launch_bounds__(NMAX) k_imp_sigma(VesIndex vi, const double* __restrict__ carry,
                                                    double* __restrict__ sigma) {
  const int v = vi.vid(blockIdx.x);
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int i = threadIdx.x;
  if (i < N) sigma[o + i] = carry[2 * o + i];
}

// ---- GMRES vector kernels over n doubles. Krylov vectors are rows of V (ld = n).

constexpr int GM_THREADS = 256;

// part[j * G + b] = CTA b's share of <V_j, w>, j < J (G = gridDim.x)
__global__ void __launch_bounds__(GM_THREADS) k_gm_dots(const double* __restrict__ V, int64_t n, int J,
                                                        const double* __restrict__ w, double* __restrict__ part) {
  __shared__ double red[GM_THREADS / 32];
  const int64_t stride = (int64_t)gridDim.x * GM_THREADS;
  for (int j = 0; j < J; ++j) {
    const double* vj = V + (int64_t)j * n;
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * GM_THREADS + threadIdx.x; e < n; e += stride) acc = fma(vj[e], w[e], acc);
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = t;
  }
}

// out[j] = sum_b part[j * G + b] in a fixed order, one warp per j; with acc non-null also acc[j] += out[j]
// (the second Gram-Schmidt pass); with norm_slot >= 0 (J = 1) out[norm_slot] = the square root instead.
__global__ void k_gm_reduce(const double* __restrict__ part, int G, int J, double* __restrict__ out,
                            double* __restrict__ acc, int norm_slot) {
  const int j = blockIdx.x;
  const int lane = threadIdx.x;
  if (j >= J) return;
  double t = 0.0;
  for (int b = lane; b < G; b += 32) t += part[(int64_t)j * G + b];
  t = warp_sum(t);
  if (lane == 0) {
    if (norm_slot >= 0) {
      out[norm_slot] = sqrt(t);
    } else {
      out[j] = t;
      if (acc) acc[j] += t;
    }
  }
}

// w -= sum_{j < J} c[j] V_j  (c: scale * coefficients, scale = -1 subtracts the projection)
__global__ void __launch_bounds__(GM_THREADS) k_gm_combine(const double* __restrict__ V, int64_t n, int J,
                                                           const double* __restrict__ c, double scale,
                                                           double* __restrict__ w) {
  const int64_t stride = (int64_t)gridDim.x * GM_THREADS;
  for (int64_t e = (int64_t)blockIdx.x * GM_THREADS + threadIdx.x; e < n; e += stride) {
    double acc = w[e];
    for (int j = 0; j < J; ++j) acc = fma(scale * c[j], V[(int64_t)j * n + e], acc);
    w[e] = acc;
  }
}

// y = a - b (elementwise)
__global__ void __launch_bounds__(GM_THREADS) k_gm_sub(const double* __restrict__ a, const double* __restrict__ b,
                                                       int64_t n, double* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * GM_THREADS;
  for (int64_t e = (int64_t)blockIdx.x * GM_THREADS + threadIdx.x; e < n; e += stride) y[e] = a[e] - b[e];
}

// y = x / *nrm (the norm read on the device); a zero norm leaves y = 0
__global__ void __launch_bounds__(GM_THREADS) k_gm_scale(const double* __restrict__ x, int64_t n,
                                                         const double* __restrict__ nrm, double* __restrict__ y) {
  const double s = *nrm > 0.0 ? 1.0 / *nrm : 0.0;
  const int64_t stride = (int64_t)gridDim.x * GM_THREADS;
  for (int64_t e = (int64_t)blockIdx.x * GM_THREADS + threadIdx.x; e < n; e += stride) y[e] = x[e] * s;
}

// y += x
__global__ void __launch_bounds__(GM_THREADS) k_gm_add(const double* __restrict__ x, int64_t n,
                                                       double* __restrict__ y) {
  const int64_t stride = (int64_t)gridDim.x * GM_THREADS;
  for (int64_t e = (int64_t)blockIdx.x * GM_THREADS + threadIdx.x; e < n; e += stride) y[e] += x[e];
}

}  // namespace vs
