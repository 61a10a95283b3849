// Mixed-precision per-vesicle solves: FP32 factorisations precondition FP64 iterative refinement
// whose residuals apply the FP64 operators without forming them (Eqs. advection_disc,
// relaxation_disc, tension_disc). One CTA per vesicle.
//
// FP64 operator actions (vectors in shared memory):
//   D_s u = diag(1/|X_alpha|) D_alpha u          (circulant, Sec. 2.2.1)
//   Ten s = [D_s(s x_s); D_s(s y_s)],  T s = S Ten s,  P v = x_s D_s v_x + y_s D_s v_y,  L s = P T s
//   B x = -kappa S [D_s^4 x_x; D_s^4 x_y]
// Solves:
//   L s = g        s <- s + Li32 (g - L s)
//   relaxation, coupled in (x, sigma):  x - dt (B x + T sigma) = X*,  P (B x + T sigma) = 0;
//     with v = S(-kappa D^4 x + Ten sigma): r1 = X* - x + dt v, r2 = -P v,
//     y = Li32 r2, dx = Ai32 (r1 + dt T32 y), dsigma = y - W32 dx   (W32 = Li32 P B32,
//     A32 = I - dt (B32 - T32 W32)): the exact block elimination of the FP32 system.
// Li32 and Ai32 are explicit FP32 inverses (k_gj_inverse), so every correction is a few FP32
// mat-vecs that all warps share. Each refinement stops at the rounding floor of its iterate
// (mp_done; at most MP_MAXIT steps); an update above 1e-11 of the iterate at the end sets ERR_REFINE.
#pragma once
#include "common.cuh"
#include "k_dense.cuh"

namespace vs {

constexpr int MP_MAXIT = 10;
constexpr int MP_THREADS = 128;  // small CTAs: many vesicles per SM hide the global-memory latency
enum : unsigned { ERR_REFINE = 32u };

__device__ inline double block_max_abs(double v, double* red) {
  v = fabs(v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  return m;
}

struct MpShared {
  double d[NMAX], sa[NMAX], tx[NMAX], ty[NMAX];
  double t0[2 * NMAX], t1[2 * NMAX], t2[2 * NMAX], red[8];
  float f0[2 * NMAX], f1[2 * NMAX];
};

// y (+)= alpha M x in FP32 for a rows x cols row-major FP32 matrix (global, read-only): each warp
// takes four rows at a time so that their loads are in flight together; ends synchronised.
__device__ inline void matvec32f(const float* __restrict__ M, int rows, int cols, const float* x, float* y,
                                 float alpha, bool add) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = 4 * wid; r0 < rows; r0 += 4 * nw) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int k = lane; k < cols; k += 32) {
      const float xk = x[k];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (r0 + q < rows) acc[q] = fmaf(__ldg(M + (int64_t)(r0 + q) * cols + k), xk, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float a = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0 && r0 + q < rows) y[r0 + q] = add ? y[r0 + q] + alpha * a : alpha * a;
    }
  }
  __syncthreads();
}

// Convergence test of a refinement: stop once the update is at the rounding floor of the iterate
// (below 4e-15 of it) or has stopped shrinking after falling below 1e-12 of it.
__device__ __forceinline__ bool mp_done(double upd, double prev, double top) {
  return upd <= 4e-15 * top || (upd <= 1e-12 * top && upd >= 0.5 * prev);
}

__device__ inline void mp_load_geom(MpShared& sh, const double* tab, const double* sa, const double* tx,
                                    const double* ty, int N, int64_t o) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sh.d[i] = tab[i];
    sh.sa[i] = sa[o + i];
    sh.tx[i] = tx[o + i];
    sh.ty[i] = ty[o + i];
  }
  __syncthreads();
}

// out[i] = D_s in (i < N); in and out distinct; ends synchronised
__device__ inline void mp_ds(const MpShared& sh, const double* in, double* out, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) out[i] = circ_row(sh.d, in, N, i) / sh.sa[i];
  __syncthreads();
}

// w = S u for the 2N x 2N row-major FP64 matrix S (global, read-only), four rows per warp pass;
// ends synchronised
__device__ inline void mp_smatvec(const double* __restrict__ S, const double* u, double* w, int n2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = 4 * wid; r0 < n2; r0 += 4 * nw) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
    for (int k = lane; k < n2; k += 32) {
      const double uk = u[k];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (r0 + q < n2) acc[q] = fma(__ldg(S + (int64_t)(r0 + q) * n2 + k), uk, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double a = warp_sum(acc[q]);
      if (lane == 0 && r0 + q < n2) w[r0 + q] = a;
    }
  }
  __syncthreads();
}

// out[c N + i] = D_s in[c N + i] for both components c = 0, 1 at once; ends synchronised
__device__ inline void mp_ds2(const MpShared& sh, const double* in, double* out, int N) {
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
    const int c = (r >= N) ? 1 : 0, i = r - c * N;
    out[r] = circ_row(sh.d, in + c * N, N, i) / sh.sa[i];
  }
  __syncthreads();
}

// out (2N) = Ten s; uses sh.t2 as scratch
__device__ inline void mp_ten(MpShared& sh, const double* s, double* out, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sh.t2[i] = s[i] * sh.tx[i];
    sh.t2[N + i] = s[i] * sh.ty[i];
  }
  __syncthreads();
  mp_ds2(sh, sh.t2, out, N);
}

// out (N) = P v
__device__ inline void mp_p(const MpShared& sh, const double* v, double* out, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    out[i] = (sh.tx[i] * circ_row(sh.d, v, N, i) + sh.ty[i] * circ_row(sh.d, v + N, N, i)) / sh.sa[i];
  __syncthreads();
}

// Solve L s = g (FP64 accuracy) with the FP32 inverse of L and FP64 matrix-free L. g is read only.
// s, e (N each), q, w (2N each) are caller shared arrays; uses sh.t2.
__device__ bool mp_solve_L(MpShared& sh, const double* S, const float* Linv, const double* g, double* s,
                           double* e, double* q, double* w, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) { s[i] = 0.0; e[i] = g[i]; }
  __syncthreads();
  double upd = 1e300, top = 0.0;
  for (int it = 0; it < MP_MAXIT; ++it) {
    if (it > 0) {
      mp_ten(sh, s, q, N);
      mp_smatvec(S, q, w, 2 * N);
      mp_p(sh, w, e, N);
      for (int i = threadIdx.x; i < N; i += blockDim.x) e[i] = g[i] - e[i];
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh.f1[i] = (float)e[i];
    __syncthreads();
    matvec32f(Linv, N, N, sh.f1, sh.f0, 1.f, false);
    double du = 0.0, sv = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      s[i] += (double)sh.f0[i];
      du = fmax(du, fabs((double)sh.f0[i]));
      sv = fmax(sv, fabs(s[i]));
    }
    const double prev = upd;
    upd = block_max_abs(du, sh.red);
    top = block_max_abs(sv, sh.red);
    if (it > 0 && mp_done(upd, prev, top)) break;
  }
  return upd <= 1e-11 * top || top == 0.0;
}

// X* = X^n + dt (u - T L^{-1} P u): (I - M^n) u with S (FP64) and Li32 cached at slot s.
__global__ void __launch_bounds__(MP_THREADS) k_advect_mp(VesIndex vi, const double* __restrict__ xy,
                                                   const double* __restrict__ u, const double* __restrict__ sa,
                                                   const double* __restrict__ tx, const double* __restrict__ ty,
                                                   const double* __restrict__ tab, const double* __restrict__ scratch,
                                                   const float* __restrict__ scratch32, int s, double dt,
                                                   double* __restrict__ xy_out, unsigned* err) {
  __shared__ MpShared sh;
  __shared__ double ub[2 * NMAX], g[NMAX], sg[NMAX], e[NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int64_t NN = (int64_t)N * N;
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) ub[r] = u[2 * o + r];
  __syncthreads();
  mp_p(sh, ub, g, N);
  const double* S = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * NN;
  const float* Linv = scratch32 + vi.moff[v] + (MatLayout::slot(s) + MatLayout::L) * NN;
  const bool ok = mp_solve_L(sh, S, Linv, g, sg, e, sh.t0, sh.t1, N);
  mp_ten(sh, sg, sh.t0, N);
  mp_smatvec(S, sh.t0, sh.t1, 2 * N);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) xy_out[2 * o + r] = xy[2 * o + r] + dt * (ub[r] - sh.t1[r]);
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

// sigma = -L^{-1} P (B X + u) at slot s (Eq. tension_disc), B X = -kappa S X_ssss.
__global__ void __launch_bounds__(MP_THREADS) k_tension_mp(VesIndex vi, const double* __restrict__ bx,
                                                    const double* __restrict__ by, const double* __restrict__ u,
                                                    const double* __restrict__ sa, const double* __restrict__ tx,
                                                    const double* __restrict__ ty, const double* __restrict__ tab,
                                                    const double* __restrict__ scratch,
                                                    const float* __restrict__ scratch32, int s, double kappa,
                                                    double* __restrict__ sigma, unsigned* err) {
  __shared__ MpShared sh;
  __shared__ double b2[2 * NMAX], g[NMAX], sg[NMAX], e[NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int64_t NN = (int64_t)N * N;
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    b2[i] = bx[o + i];
    b2[N + i] = by[o + i];
  }
  __syncthreads();
  const double* S = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * NN;
  mp_smatvec(S, b2, sh.t0, 2 * N);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.t0[r] = -kappa * sh.t0[r] + u[2 * o + r];
  __syncthreads();
  mp_p(sh, sh.t0, g, N);
  const float* Linv = scratch32 + vi.moff[v] + (MatLayout::slot(s) + MatLayout::L) * NN;
  const bool ok = mp_solve_L(sh, S, Linv, g, sg, e, sh.t0, sh.t1, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sigma[o + i] = -sg[i];
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

// Relaxation (Eq. relaxation_disc) by refinement of the coupled (x, sigma) system at slot s.
__global__ void __launch_bounds__(MP_THREADS) k_relax_mp(VesIndex vi, const double* __restrict__ xy_star,
                                                  const double* __restrict__ sa, const double* __restrict__ tx,
                                                  const double* __restrict__ ty, const double* __restrict__ tab,
                                                  const double* __restrict__ scratch,
                                                  const float* __restrict__ scratch32, int s, int64_t ainv_sub,
                                                  double kappa, double dt, double* __restrict__ xy_out,
                                                  unsigned* err) {
  __shared__ MpShared sh;
  __shared__ double b[2 * NMAX], x[2 * NMAX], sg[NMAX], r1[2 * NMAX], y2[NMAX];
  __shared__ float fy[NMAX], fr[2 * NMAX], fdx[2 * NMAX], fw[NMAX];
  const int v = blockIdx.x;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int64_t NN = (int64_t)N * N;
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) { b[r] = xy_star[2 * o + r]; x[r] = 0.0; }
  for (int i = threadIdx.x; i < N; i += blockDim.x) sg[i] = 0.0;
  __syncthreads();
  const double* S = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::S) * NN;
  const float* base32 = scratch32 + vi.moff[v];
  const float* T32 = base32 + (MatLayout::slot(s) + MatLayout::T) * NN;
  const float* Linv = base32 + (MatLayout::slot(s) + MatLayout::L) * NN;  // Li32
  const float* W32 = base32 + MatLayout::W * NN;
  const float* Ainv = base32 + ainv_sub * NN;                              // Ai32
  double upd = 1e300, top = 0.0;
  for (int it = 0; it < MP_MAXIT; ++it) {
    if (it == 0) {
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) r1[r] = b[r];
      for (int i = threadIdx.x; i < N; i += blockDim.x) y2[i] = 0.0;
      __syncthreads();
    } else {
      // q = -kappa D^4 x + Ten sigma  (into sh.t0), v = S q (into sh.t1)
      mp_ds2(sh, x, sh.t1, N);
      mp_ds2(sh, sh.t1, sh.t2, N);
      mp_ds2(sh, sh.t2, sh.t1, N);
      mp_ds2(sh, sh.t1, sh.t0, N);
      mp_ten(sh, sg, sh.t1, N);
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.t0[r] = -kappa * sh.t0[r] + sh.t1[r];
      __syncthreads();
      mp_smatvec(S, sh.t0, sh.t1, 2 * N);
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) r1[r] = b[r] - x[r] + dt * sh.t1[r];
      __syncthreads();
      mp_p(sh, sh.t1, y2, N);
      for (int i = threadIdx.x; i < N; i += blockDim.x) y2[i] = -y2[i];
      __syncthreads();
    }
    // correction in FP32: y = Li32 r2, dx = Ai32 (r1 + dt T32 y), dsigma = y - W32 dx
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh.f0[i] = (float)y2[i];
    for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) fr[r] = (float)r1[r];
    __syncthreads();
    matvec32f(Linv, N, N, sh.f0, fy, 1.f, false);
    matvec32f(T32, 2 * N, N, fy, fr, (float)dt, true);
    matvec32f(Ainv, 2 * N, 2 * N, fr, fdx, 1.f, false);
    matvec32f(W32, N, 2 * N, fdx, fw, 1.f, false);
    double du = 0.0, xv = 0.0;
    for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
      x[r] += (double)fdx[r];
      du = fmax(du, fabs((double)fdx[r]));
      xv = fmax(xv, fabs(x[r]));
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) sg[i] += (double)fy[i] - (double)fw[i];
    const double prev = upd;
    upd = block_max_abs(du, sh.red);
    top = block_max_abs(xv, sh.red);
    if (it > 0 && mp_done(upd, prev, top)) break;
  }
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) xy_out[2 * o + r] = x[r];
  if (!(upd <= 1e-11 * top) && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

}  // namespace vs
