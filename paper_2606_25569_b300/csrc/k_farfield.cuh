// All-pairs far-field single-layer sum (Sec. 2.2.2, Sec. 4.1, Algorithm 4).
//
// u(x_i) += sum over source vesicles v != vesicle(i), v not near x_i, of
//           sum_j [ -log|r| g_j + (r . g_j) r / |r|^2 ],  r = x_i - X_vj,
// g_j = f_j |X_alpha|_j (2 pi / N_v) / (4 pi mu) (trapezoid rule with the 2D Stokeslet).
// x_i is near v when min_j |r|^2 <= h_v^2, h_v = L_v / N_v; its pair is then skipped and the
// source vesicle recorded in the target's near list (ascending v, at most MAX_NEAR). The minimum is
// only tracked for targets inside a conservative reach circle of v (a bound from its radius).
//
// FP32 path: each source carries its offset from its vesicle's centre c_v; per (target, source
// vesicle) the centre difference is formed once from float hi/lo splits, so |r| keeps relative
// accuracy for close pairs in a large box. Per-vesicle partial sums are FP32 and are added to the
// running total with Neumaier compensation. -log|r| = -(ln 2 / 2) log2(|r|^2), with lg2 and rcp on
// the special-function unit.
//
// One thread per target; source vesicles are staged through shared memory in chunks of whole
// vesicles (chunk boundaries precomputed on the host, at most CHUNK points each). THREADS and CHUNK
// only change the launch shape and the staging: every target sums the same terms in the same order
// (vesicles ascending), so all instantiations give bitwise identical results (autotuned per suspension).
#pragma once
#include "common.cuh"

namespace vs {

constexpr int FF_THREADS = 128;  // default launch shape (far-field plans, the allocation-free entry point)
constexpr int FF_CHUNK = 2048;

__device__ __forceinline__ float fast_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void neumaier_add(float& s, float& c, float p) {
  const float t = s + p;
  c += (fabsf(s) >= fabsf(p)) ? ((s - t) + p) : ((p - t) + s);
  s = t;
}

// Sum over the sources j0..j1-1 (shared memory) of one vesicle for the target at (qx, qy) in the
// vesicle's frame; with MIN the smallest |r|^2 is tracked too.
template <bool MIN>
__device__ __forceinline__ void ff_sum(const float4* sh, int j0, int j1, float qx, float qy, float& ax, float& ay,
                                       float& lx, float& ly, float& mn) {
#pragma unroll 16
  for (int j = j0; j < j1; ++j) {
    const float4 s = sh[j];
    const float rx = qx - s.x, ry = qy - s.y;
    const float r2 = fmaf(rx, rx, ry * ry);
    if (MIN) mn = fminf(mn, r2);
    const float lg = fast_lg2(r2);
    const float inv = fast_rcp(r2);
    lx = fmaf(lg, s.z, lx);
    ly = fmaf(lg, s.w, ly);
    const float q = fmaf(rx, s.z, ry * s.w) * inv;
    ax = fmaf(q, rx, ax);
    ay = fmaf(q, ry, ay);
  }
}

struct FarFieldArgs {
  int64_t P;                 // total points (targets = sources)
  int M;
  const int32_t* owner;      // vesicle of each point [P]
  const int64_t* voff;       // point offsets [M+1]
  const int32_t* chunk;      // chunk boundaries in vesicles [nchunk+1]
  int nchunk;
  int near_mask;             // 1: skip and record near pairs
  double* u;                 // accumulated into (+=), CSR blocks [u_x(N), u_y(N)] per vesicle
  int* near_cnt;             // [P] (written when near_mask)
  int* near_v;               // [P * MAX_NEAR]
  unsigned* err;
};

template <int THREADS, int CHUNK>
__global__ void __launch_bounds__(THREADS) k_farfield_f32(FarFieldArgs a, const float4* __restrict__ src,
                                                          const float4* __restrict__ centre32,
                                                          const float2* __restrict__ h2) {
  __shared__ float4 sh[CHUNK];
  const int64_t t = (int64_t)blockIdx.x * THREADS + threadIdx.x;
  const bool valid = t < a.P;
  const int tv = valid ? a.owner[t] : -1;
  const float4 ts = valid ? src[t] : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 tc = valid ? centre32[tv] : make_float4(0.f, 0.f, 0.f, 0.f);
  float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
  int ncnt = 0;
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2
  for (int c = 0; c < a.nchunk; ++c) {
    const int v0 = a.chunk[c], v1 = a.chunk[c + 1];
    const int64_t p0 = a.voff[v0], p1 = a.voff[v1];
    __syncthreads();
    for (int64_t q = p0 + threadIdx.x; q < p1; q += THREADS) sh[q - p0] = src[q];
    __syncthreads();
    if (!valid) continue;
    for (int sv = v0; sv < v1; ++sv) {
      if (sv == tv) continue;
      const float4 sc = centre32[sv];
      const float qx = ((tc.x - sc.x) + (tc.z - sc.z)) + ts.x;
      const float qy = ((tc.y - sc.y) + (tc.w - sc.w)) + ts.y;
      const int j0 = (int)(a.voff[sv] - p0), j1 = (int)(a.voff[sv + 1] - p0);
      const float2 nr = h2[sv];
      // the minimum distance is only needed when the target lies within reach of the vesicle
      const bool test = a.near_mask && fmaf(qx, qx, qy * qy) <= nr.y;
      float ax = 0.f, ay = 0.f, lx = 0.f, ly = 0.f, mn = 3.0e38f;
      if (test)
        ff_sum<true>(sh, j0, j1, qx, qy, ax, ay, lx, ly, mn);
      else
        ff_sum<false>(sh, j0, j1, qx, qy, ax, ay, lx, ly, mn);
      if (test && mn <= nr.x) {
        if (ncnt < MAX_NEAR) a.near_v[t * MAX_NEAR + ncnt] = sv;
        else atomicOr(a.err, ERR_NEAR_OVERFLOW);
        ++ncnt;
      } else {
        neumaier_add(sx, cx, fmaf(hl2, lx, ax));
        neumaier_add(sy, cy, fmaf(hl2, ly, ay));
      }
    }
  }
  if (valid) {
    const int64_t to = a.voff[tv];
    const int tN = (int)(a.voff[tv + 1] - to);
    a.u[2 * to + (t - to)] += (double)sx + (double)cx;
    a.u[2 * to + tN + (t - to)] += (double)sy + (double)cy;
    if (a.near_mask) a.near_cnt[t] = ncnt < MAX_NEAR ? ncnt : MAX_NEAR;
  }
}

// FP64 reference-precision variant (absolute coordinates, log and division in FP64).
__global__ void __launch_bounds__(FF_THREADS) k_farfield_f64(FarFieldArgs a, const double* __restrict__ xy,
                                                             const double* __restrict__ g64,
                                                             const double* __restrict__ length,
                                                             const int32_t* __restrict__ Nv) {
  const int64_t t = (int64_t)blockIdx.x * FF_THREADS + threadIdx.x;
  if (t >= a.P) return;
  const int tv = a.owner[t];
  const int64_t to = a.voff[tv];
  const int tN = Nv[tv];
  const double tx = xy[2 * to + (t - to)];
  const double ty = xy[2 * to + tN + (t - to)];
  double sx = 0.0, sy = 0.0;
  int ncnt = 0;
  for (int sv = 0; sv < a.M; ++sv) {
    if (sv == tv) continue;
    const int64_t so = a.voff[sv];
    const int sN = Nv[sv];
    double ax = 0.0, ay = 0.0, mn = 1.0e300;
    for (int j = 0; j < sN; ++j) {
      const double rx = tx - xy[2 * so + j], ry = ty - xy[2 * so + sN + j];
      const double r2 = rx * rx + ry * ry;
      mn = fmin(mn, r2);
      const double lg = -0.5 * log(r2);
      const double g1 = g64[2 * so + j], g2 = g64[2 * so + sN + j];
      const double q = (rx * g1 + ry * g2) / r2;
      ax += lg * g1 + q * rx;
      ay += lg * g2 + q * ry;
    }
    const double h = length[sv] / sN;
    if (a.near_mask && mn <= h * h) {
      if (ncnt < MAX_NEAR) a.near_v[t * MAX_NEAR + ncnt] = sv;
      else atomicOr(a.err, ERR_NEAR_OVERFLOW);
      ++ncnt;
    } else {
      sx += ax;
      sy += ay;
    }
  }
  a.u[2 * to + (t - to)] += sx;
  a.u[2 * to + tN + (t - to)] += sy;
  if (a.near_mask) a.near_cnt[t] = ncnt < MAX_NEAR ? ncnt : MAX_NEAR;
}

}  // namespace vs
