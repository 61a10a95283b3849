// Mixed-precision per-vesicle solves: explicit FP32 inverses precondition iterative refinement whose
// residuals apply the operators of Eqs. advection_disc, relaxation_disc and tension_disc without
// forming them, in double-float arithmetic (FP64 runs at 1/64 of the FP32 rate on this part). One CTA
// per vesicle.
//
// Operator actions (vectors in shared memory, double-float):
//   D_s u = diag(1/|X_alpha|) D_alpha u          (circulant, Sec. 2.2.1)
//   Ten s = [D_s(s x_s); D_s(s y_s)],  T s = S Ten s,  P v = x_s D_s v_x + y_s D_s v_y,  L s = P T s
//   B x = -kappa S [D_s^4 x_x; D_s^4 x_y]
// with S = S_hi + S_lo, the FP64 self matrix split into two FP32 matrices by k_self_matrix.
// Solves:
//   L s = g        s <- s + Li32 (g - L s)
//   relaxation, coupled in (x, sigma):  x - dt (B x + T sigma) = X*,  P (B x + T sigma) = 0;
//     with v = S(-kappa D^4 x + Ten sigma): r1 = X* - x + dt v, r2 = -P v,
//     y = Li32 r2, dx = Ai32 (r1 + dt T32 y), dsigma = y - W32 dx   (W32 = Li32 P B32,
//     A32 = I - dt (B32 - T32 W32)): the exact block elimination of the FP32 system.
// Li32 and Ai32 are explicit FP32 inverses (k_gj_inverse), so every correction is a few FP32 mat-vecs
// that all warps share. Iterates are kept in FP64. Each refinement stops once the error estimated from its
// contraction is below MP_LEFT of the iterate or its update reaches the rounding floor of the residual
// arithmetic (mp_done; at most MP_MAXIT steps); an estimated error above MP_FAIL at the end sets ERR_REFINE.
#pragma once
#include "common.cuh"
#include "k_dense.cuh"
#include "dfloat.cuh"

namespace vs {

constexpr int MP_MAXIT = 10;
// CTA sizes of the refinement kernels: 128 threads when there are many vesicles per SM to hide the
// memory latency, 256 when a few large vesicles leave the SMs short of work (mp_threads)
constexpr int MP_THREADS = 128, MP_THREADS_WIDE = 256;
constexpr float MP_FLOOR = 1e-14f, MP_STALL = 1e-11f, MP_FAIL = 1e-10f, MP_LEFT = 1e-13f;
enum : unsigned { ERR_REFINE = 32u };

// Block-wide maximum of |v| in FP32 (the stop rule's magnitudes; the FP64 pipe runs at 1/64 of the FP32
// rate on this part); red holds one float per warp. All threads get it.
__device__ inline float block_max_absf(float v, float* red) {
  v = fabsf(v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  return m;
}

struct MpShared {
  float2 d[NMAX], is[NMAX], tx[NMAX], ty[NMAX];   // D_alpha circulant, 1/|X_alpha|, x_s, y_s
  float2 u0[2 * NMAX], u1[2 * NMAX], u2[2 * NMAX]; // double-float work vectors
  double red[8];
  float redf[8];
  __align__(16) float f0[2 * NMAX];                // FP32 corrections
  __align__(16) float f1[2 * NMAX];
};

// y (+)= alpha M x in FP32 for a rows x cols row-major FP32 matrix (global, read-only; cols even, at most
// COLS, 128 or 256). Each warp takes MV_ROWS rows at a time and each lane two adjacent columns per 64, all loads
// of a pass issued before the arithmetic so that enough bytes are in flight to cover the memory latency;
// ends synchronised. x must be 8-byte aligned.
constexpr int MV_ROWS = 4;
template <int COLS>
__device__ inline void matvec32f(const float* __restrict__ M, int rows, int cols, const float* x, float* y,
                                 float alpha, bool add) {
  if ((cols & 3) == 0 && ((reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(x)) & 15) == 0) {
    // one row per thread, the row read as float4 and x broadcast from shared memory: no cross-lane reduction
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      const float4* Mr = reinterpret_cast<const float4*>(M + (int64_t)r * cols);
      float a0 = 0.f, a1 = 0.f;
#pragma unroll 8
      for (int k = 0; k < cols / 4; ++k) {
        const float4 m = __ldg(Mr + k);
        const float4 xv = x4[k];
        a0 = fmaf(m.x, xv.x, a0);
        a1 = fmaf(m.y, xv.y, a1);
        a0 = fmaf(m.z, xv.z, a0);
        a1 = fmaf(m.w, xv.w, a1);
      }
      const float a = a0 + a1;
      y[r] = add ? y[r] + alpha * a : alpha * a;
    }
    __syncthreads();
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = MV_ROWS * wid; r0 < rows; r0 += MV_ROWS * nw) {
    float2 mv[COLS / 64][MV_ROWS];
#pragma unroll
    for (int t = 0; t < COLS / 64; ++t) {
      const int k = 2 * lane + 64 * t;
#pragma unroll
      for (int q = 0; q < MV_ROWS; ++q)
        mv[t][q] = (k < cols && r0 + q < rows)
                       ? __ldg(reinterpret_cast<const float2*>(M + (int64_t)(r0 + q) * cols + k))
                       : make_float2(0.f, 0.f);
    }
    float acc[MV_ROWS];
#pragma unroll
    for (int q = 0; q < MV_ROWS; ++q) acc[q] = 0.f;
#pragma unroll
    for (int t = 0; t < COLS / 64; ++t) {
      const int k = 2 * lane + 64 * t;
      if (k < cols) {
        const float2 xk = *reinterpret_cast<const float2*>(x + k);
#pragma unroll
        for (int q = 0; q < MV_ROWS; ++q) acc[q] = fmaf(mv[t][q].y, xk.y, fmaf(mv[t][q].x, xk.x, acc[q]));
      }
    }
#pragma unroll
    for (int q = 0; q < MV_ROWS; ++q) {
      float a = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (lane == 0 && r0 + q < rows) y[r0 + q] = add ? y[r0 + q] + alpha * a : alpha * a;
    }
  }
  __syncthreads();
}

// Error left in the iterate after an update of size upd that followed one of size prev, for an iteration
// that contracts at the observed rate upd / prev: upd^2 / prev (and at most upd).
__device__ __forceinline__ float mp_left(float upd, float prev) { return fminf(upd, upd * (upd / prev)); }

// Convergence test of a refinement: stop once the estimated error left is below MP_LEFT of the iterate
// (with FP32 inverses contracting by about 3e-7 a step this is after the first residual step), or the
// update is below MP_FLOOR, or has stopped shrinking after falling below MP_STALL (the rounding floor of
// the residual arithmetic).
// The magnitudes are FP32 maxima of the FP32 corrections; the iterate's size `top` is taken from the first
// correction (the iterate starts at zero, and later corrections change it by a few 1e-7 of itself).
__device__ __forceinline__ bool mp_done(float upd, float prev, float top) {
  return mp_left(upd, prev) <= MP_LEFT * top || upd <= MP_FLOOR * top || (upd <= MP_STALL * top && upd >= 0.5f * prev);
}

__device__ inline void mp_load_geom(MpShared& sh, const double* tab, const double* sa, const double* tx,
                                    const double* ty, int N, int64_t o) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sh.d[i] = df_of(tab[i]);
    sh.is[i] = df_of(1.0 / sa[o + i]);
    sh.tx[i] = df_of(tx[o + i]);
    sh.ty[i] = df_of(ty[o + i]);
  }
  __syncthreads();
}

// out[c N + i] = D_s in[c N + i] for both components c = 0, 1; in and out distinct; ends synchronised
__device__ inline void mp_ds2(const MpShared& sh, const float2* in, float2* out, int N) {
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
    const int c = (r >= N) ? 1 : 0, i = r - c * N;
    out[r] = df_mul(circ_df(sh.d, in + c * N, N, i), sh.is[i]);
  }
  __syncthreads();
}

// out (2N) = Ten s; uses sh.u2 as scratch
__device__ inline void mp_ten(MpShared& sh, const float2* s, float2* out, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sh.u2[i] = df_mul(s[i], sh.tx[i]);
    sh.u2[N + i] = df_mul(s[i], sh.ty[i]);
  }
  __syncthreads();
  mp_ds2(sh, sh.u2, out, N);
}

// out (N) = P v; ends synchronised
__device__ inline void mp_p(const MpShared& sh, const float2* v, float2* out, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const float2 a = df_mul(sh.tx[i], circ_df(sh.d, v, N, i));
    const float2 b = df_mul(sh.ty[i], circ_df(sh.d, v + N, N, i));
    out[i] = df_mul(df_add(a, b), sh.is[i]);
  }
  __syncthreads();
}

// w = S u for the 2N x 2N matrix S = Sh + Sl (two row-major FP32 matrices in global memory): MV_ROWS
// rows per warp pass, each lane two adjacent columns per 64 (all loads of a pass issued first), partial
// sums merged across the warp; ends synchronised
template <int COLS>
__device__ inline void mp_smatvec(const float* __restrict__ Sh, const float* __restrict__ Sl, const float2* u,
                                  float2* w, int n2) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r0 = MV_ROWS * wid; r0 < n2; r0 += MV_ROWS * nw) {
    float2 hv[COLS / 64][MV_ROWS], lv[COLS / 64][MV_ROWS];
#pragma unroll
    for (int t = 0; t < COLS / 64; ++t) {
      const int k = 2 * lane + 64 * t;
#pragma unroll
      for (int q = 0; q < MV_ROWS; ++q) {
        const bool in = k < n2 && r0 + q < n2;
        const int64_t e = (int64_t)(r0 + q) * n2 + k;
        hv[t][q] = in ? __ldg(reinterpret_cast<const float2*>(Sh + e)) : make_float2(0.f, 0.f);
        lv[t][q] = in ? __ldg(reinterpret_cast<const float2*>(Sl + e)) : make_float2(0.f, 0.f);
      }
    }
    Dot2 acc[MV_ROWS];
#pragma unroll
    for (int t = 0; t < COLS / 64; ++t) {
      const int k = 2 * lane + 64 * t;
      if (k < n2) {
        const float2 u0 = u[k], u1 = u[k + 1];
#pragma unroll
        for (int q = 0; q < MV_ROWS; ++q) {
          acc[q].add(make_float2(hv[t][q].x, lv[t][q].x), u0);
          acc[q].add(make_float2(hv[t][q].y, lv[t][q].y), u1);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < MV_ROWS; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, acc[q].s, o);
        const float c2 = __shfl_xor_sync(0xffffffffu, acc[q].c, o);
        acc[q].merge(s2, c2);
      }
      if (lane == 0 && r0 + q < n2) w[r0 + q] = acc[q].value();
    }
  }
  __syncthreads();
}

// The FP32 blocks of vesicle v at slot s: S_hi, S_lo, T32, Li32
struct MpMats {
  const float *sh, *sl, *t32, *li;
};
__device__ __forceinline__ MpMats mp_mats(const VesIndex& vi, const float* scratch32, int v, int s) {
  const int N = vi.N[v];
  const int64_t NN = (int64_t)N * N;
  const float* b = scratch32 + vi.moff[v];
  return MpMats{b + (MatLayout::slot(s) + MatLayout::S) * NN, b + (MatLayout::slot(s) + MatLayout::SL) * NN,
                b + (MatLayout::slot(s) + MatLayout::T) * NN, b + (MatLayout::slot(s) + MatLayout::L) * NN};
}

// Solve L s = g (s FP64, g double-float and read only) with Li32 and the matrix-free L.
// e (N) and q, w (2N) are caller shared double-float arrays; uses sh.u2, sh.f0, sh.f1.
template <int COLS>
__device__ bool mp_solve_L(MpShared& sh, const MpMats& m, const float2* g, double* s, float2* e, float2* q,
                           float2* w, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) { s[i] = 0.0; e[i] = g[i]; }
  __syncthreads();
  float upd = 3e38f, top = 0.f, prev_upd = 3e38f;
  for (int it = 0; it < MP_MAXIT; ++it) {
    if (it > 0) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) w[i] = df_of(s[i]);
      __syncthreads();
      mp_ten(sh, w, q, N);
      mp_smatvec<COLS>(m.sh, m.sl, q, w, 2 * N);
      mp_p(sh, w, e, N);
      for (int i = threadIdx.x; i < N; i += blockDim.x) e[i] = df_add(g[i], make_float2(-e[i].x, -e[i].y));
      __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh.f1[i] = e[i].x;
    __syncthreads();
    matvec32f<COLS>(m.li, N, N, sh.f1, sh.f0, 1.f, false);
    float du = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      s[i] += (double)sh.f0[i];
      du = fmaxf(du, fabsf(sh.f0[i]));
    }
    const float prev = upd;
    upd = block_max_absf(du, sh.redf);
    if (it == 0) top = upd;  // s = the first correction
    prev_upd = prev;
    if (it > 0 && mp_done(upd, prev, top)) break;
  }
  return mp_left(upd, prev_upd) <= MP_FAIL * top || top == 0.f;
}

// X* = X^n + dt (u - T L^{-1} P u): (I - M^n) u with the operators cached at slot s.
template <int THREADS, int COLS>
__global__ void __launch_bounds__(THREADS) k_advect_mp(VesIndex vi, const double* __restrict__ xy,
                                                   const double* __restrict__ u, const double* __restrict__ sa,
                                                   const double* __restrict__ tx, const double* __restrict__ ty,
                                                   const double* __restrict__ tab,
                                                   const float* __restrict__ scratch32, int s, double dt,
                                                   double* __restrict__ xy_out, unsigned* err,
                                                   const int* __restrict__ active = nullptr) {
  __shared__ MpShared sh;
  __shared__ float2 g[NMAX], e[NMAX];
  __shared__ double sg[NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.u0[r] = df_of(u[2 * o + r]);
  __syncthreads();
  mp_p(sh, sh.u0, g, N);
  const MpMats m = mp_mats(vi, scratch32, v, s);
  const bool ok = mp_solve_L<COLS>(sh, m, g, sg, e, sh.u1, sh.u0, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) e[i] = df_of(sg[i]);
  __syncthreads();
  mp_ten(sh, e, sh.u1, N);
  mp_smatvec<COLS>(m.sh, m.sl, sh.u1, sh.u0, 2 * N);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x)
    xy_out[2 * o + r] = xy[2 * o + r] + dt * (u[2 * o + r] - df_val(sh.u0[r]));
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

// sigma = -L^{-1} P (B X + u) at slot s (Eq. tension_disc), B X = -kappa S X_ssss.
template <int THREADS, int COLS>
__global__ void __launch_bounds__(THREADS) k_tension_mp(VesIndex vi, const double* __restrict__ bx,
                                                    const double* __restrict__ by, const double* __restrict__ u,
                                                    const double* __restrict__ sa, const double* __restrict__ tx,
                                                    const double* __restrict__ ty, const double* __restrict__ tab,
                                                    const float* __restrict__ scratch32, int s, double kappa,
                                                    double* __restrict__ sigma, unsigned* err,
                                                    const int* __restrict__ active = nullptr) {
  __shared__ MpShared sh;
  __shared__ float2 g[NMAX], e[NMAX];
  __shared__ double sg[NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    sh.u0[i] = df_of(bx[o + i]);
    sh.u0[N + i] = df_of(by[o + i]);
  }
  __syncthreads();
  const MpMats m = mp_mats(vi, scratch32, v, s);
  mp_smatvec<COLS>(m.sh, m.sl, sh.u0, sh.u1, 2 * N);
  const float2 mk = df_of(-kappa);
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.u1[r] = df_add(df_mul(mk, sh.u1[r]), df_of(u[2 * o + r]));
  __syncthreads();
  mp_p(sh, sh.u1, g, N);
  const bool ok = mp_solve_L<COLS>(sh, m, g, sg, e, sh.u1, sh.u0, N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) sigma[o + i] = -sg[i];
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

// Relaxation (Eq. relaxation_disc) by refinement of the coupled (x, sigma) system at slot s. The
// iterate x is kept relative to the mean point of X* (the operators only see its derivatives).
template <int THREADS, int COLS>
__global__ void __launch_bounds__(THREADS) k_relax_mp(VesIndex vi, const double* __restrict__ xy_star,
                                                  const double* __restrict__ sa, const double* __restrict__ tx,
                                                  const double* __restrict__ ty, const double* __restrict__ tab,
                                                  const float* __restrict__ scratch32, int s, int64_t ainv_sub,
                                                  double kappa, double dt, double* __restrict__ xy_out,
                                                  unsigned* err, const int* __restrict__ active) {
  __shared__ MpShared sh;
  __shared__ double b[2 * NMAX], x[2 * NMAX], sg[NMAX], r1[2 * NMAX], cen[2];
  __shared__ float2 y2[NMAX];
  __shared__ __align__(16) float fy[NMAX], fr[2 * NMAX], fdx[2 * NMAX], fw[NMAX];
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int64_t o = vi.off[v];
  const int64_t NN = (int64_t)N * N;
  mp_load_geom(sh, tab + vi.toff[v], sa, tx, ty, N, o);
  double mx = 0.0, my = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    mx += xy_star[2 * o + i];
    my += xy_star[2 * o + N + i];
  }
  mx = block_sum(mx, sh.red) / N;
  my = block_sum(my, sh.red) / N;
  if (threadIdx.x == 0) { cen[0] = mx; cen[1] = my; }
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
    b[r] = xy_star[2 * o + r] - ((r < N) ? mx : my);  // X* relative to its mean point
    x[r] = 0.0;
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) sg[i] = 0.0;
  __syncthreads();
  const MpMats m = mp_mats(vi, scratch32, v, s);
  const float* base32 = scratch32 + vi.moff[v];
  const float* W32 = base32 + MatLayout::W * NN;
  const float* Ainv = base32 + ainv_sub * NN;  // Ai32
  const float2 mk = df_of(-kappa);
  float upd = 3e38f, top = 0.f, prev_upd = 3e38f;
  for (int it = 0; it < MP_MAXIT; ++it) {
    if (it == 0) {
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) r1[r] = b[r];
      for (int i = threadIdx.x; i < N; i += blockDim.x) y2[i] = make_float2(0.f, 0.f);
      __syncthreads();
    } else {
      // q = -kappa D^4 x + Ten sigma (into u0), v = S q (into u1)
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.u0[r] = df_of(x[r]);
      __syncthreads();
      mp_ds2(sh, sh.u0, sh.u1, N);
      mp_ds2(sh, sh.u1, sh.u2, N);
      mp_ds2(sh, sh.u2, sh.u1, N);
      mp_ds2(sh, sh.u1, sh.u0, N);
      for (int i = threadIdx.x; i < N; i += blockDim.x) sh.u1[i] = df_of(sg[i]);
      __syncthreads();
      float2* tsg = reinterpret_cast<float2*>(r1);  // r1 is free until the residual: Ten sigma (2N) into it
      mp_ten(sh, sh.u1, tsg, N);
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) sh.u0[r] = df_add(df_mul(mk, sh.u0[r]), tsg[r]);
      __syncthreads();
      mp_smatvec<COLS>(m.sh, m.sl, sh.u0, sh.u1, 2 * N);
      for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) r1[r] = b[r] - x[r] + dt * df_val(sh.u1[r]);
      __syncthreads();
      mp_p(sh, sh.u1, y2, N);
    }
    // correction in FP32: y = Li32 r2 (r2 = -P v), dx = Ai32 (r1 + dt T32 y), dsigma = y - W32 dx
    for (int i = threadIdx.x; i < N; i += blockDim.x) sh.f0[i] = -y2[i].x;
    for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) fr[r] = (float)r1[r];
    __syncthreads();
    matvec32f<COLS>(m.li, N, N, sh.f0, fy, 1.f, false);
    matvec32f<COLS>(m.t32, 2 * N, N, fy, fr, (float)dt, true);
    matvec32f<COLS>(Ainv, 2 * N, 2 * N, fr, fdx, 1.f, false);
    matvec32f<COLS>(W32, N, 2 * N, fdx, fw, 1.f, false);
    float du = 0.f;
    for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
      x[r] += (double)fdx[r];
      du = fmaxf(du, fabsf(fdx[r]));
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) sg[i] += (double)fy[i] - (double)fw[i];
    const float prev = upd;
    upd = block_max_absf(du, sh.redf);
    if (it == 0) top = upd;  // x = the first correction
    prev_upd = prev;
    if (it > 0 && mp_done(upd, prev, top)) break;
  }
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) xy_out[2 * o + r] = x[r] + cen[r < N ? 0 : 1];
  if (!(mp_left(upd, prev_upd) <= MP_FAIL * top) && threadIdx.x == 0) atomicOr(err, ERR_REFINE);
}

}  // namespace vs
