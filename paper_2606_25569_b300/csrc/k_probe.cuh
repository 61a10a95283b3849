// FP32 throughput probes: the measured denominators of the far field's roofline. Both kernels work on
// registers only (nothing is loaded in the timed loop, nothing is exchanged between lanes), so their rate is
// the rate of their instruction stream on the FP32 pipe and the special-function unit.
//   k_probe_ffma2: eight independent chains of paired FMAs per thread (the FP32 pipe's issue limit).
//   k_probe_pair:  the arithmetic of one step of the symmetric far field's pair loop (ffs_pair2) on eight
//                  target rows against one pair of sources: per two pairs 18 paired FP32 instructions
//                  (r 2, |r|^2 2, both reactions 7 each) and 2 lg2 + 2 rcp.
#pragma once
#include "k_farfield.cuh"

namespace vs {

constexpr int PROBE_ROWS = 8;

__global__ void __launch_bounds__(256) k_probe_ffma2(float* out, int iters) {
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, (float)i);
  const float2 b = make_float2(1.0001f, 1.0002f), c = make_float2(1e-7f, 2e-7f);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = __ffma2_rn(a[i], b, c);
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_pair(float* out, int iters) {
  float2 ntx[PROBE_ROWS], nty[PROBE_ROWS], lx[PROBE_ROWS], ly[PROBE_ROWS], ax[PROBE_ROWS], ay[PROBE_ROWS];
  const float base = threadIdx.x * 1e-4f;
#pragma unroll
  for (int r = 0; r < PROBE_ROWS; ++r) {
    ntx[r] = make_float2(-0.1f * r - base, -0.2f * r - base);
    nty[r] = make_float2(0.3f * r + base, 0.05f * r + 1e-3f);
    lx[r] = ly[r] = ax[r] = ay[r] = make_float2(0.f, 0.f);
  }
  float2 sx = make_float2(1.f, 1.1f), sy = make_float2(0.7f, 0.9f), ux = make_float2(0.f, 0.f), uy = ux;
  const float2 sz = make_float2(0.3f, 0.2f), sw = make_float2(0.5f, 0.4f), t2 = make_float2(1.f, 1.f);
  const float2 gx = make_float2(0.01f, 0.01f), gy = make_float2(0.02f, 0.02f);
  const float2 rz = make_float2(0.1f, 0.1f), rw = make_float2(0.2f, 0.2f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < PROBE_ROWS; ++r) {
      const float2 rx = __ffma2_rn(sx, t2, ntx[r]), ry = __ffma2_rn(sy, t2, nty[r]);
      const float2 r2 = __ffma2_rn(rx, rx, __fmul2_rn(ry, ry));
      const float2 lg = make_float2(fast_lg2(r2.x), fast_lg2(r2.y));
      const float2 inv = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
      lx[r] = __ffma2_rn(lg, sz, lx[r]);
      ly[r] = __ffma2_rn(lg, sw, ly[r]);
      const float2 q = __fmul2_rn(__ffma2_rn(rx, sz, __fmul2_rn(ry, sw)), inv);
      ax[r] = __ffma2_rn(q, rx, ax[r]);
      ay[r] = __ffma2_rn(q, ry, ay[r]);
      ux = __ffma2_rn(lg, gx, ux);
      uy = __ffma2_rn(lg, gy, uy);
      const float2 qt = __fmul2_rn(__ffma2_rn(rx, rz, __fmul2_rn(ry, rw)), inv);
      ux = __ffma2_rn(qt, rx, ux);
      uy = __ffma2_rn(qt, ry, uy);
    }
    sx.x += 1e-6f;  // a new source pair every step
    sy.y -= 1e-6f;
  }
  float s = ux.x + ux.y + uy.x + uy.y;
#pragma unroll
  for (int r = 0; r < PROBE_ROWS; ++r) s += lx[r].x + lx[r].y + ly[r].x + ly[r].y + ax[r].x + ax[r].y + ay[r].x + ay[r].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace vs
