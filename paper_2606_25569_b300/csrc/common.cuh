// Shared definitions for the vesicle-suspension kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define VS_PI 3.14159265358979323846

namespace vs {

constexpr int NMAX = 128;          // largest points per vesicle handled by the per-vesicle kernels
constexpr int TAB_STRIDE = 18;     // table doubles per N (see tables.cuh)
constexpr int MAX_NEAR = 8;        // near source vesicles recorded per target point

// Device-side error bits, OR-ed into one word per suspension and read back by the host.
enum : unsigned {
  ERR_PIVOT = 1u,        // zero pivot in a batched LU
  ERR_NONFINITE = 2u,    // NaN / Inf in a state vector
  ERR_CORRECTION = 4u,   // area/length correction did not converge
  ERR_NEAR_OVERFLOW = 8u // a target had more than MAX_NEAR near vesicles
};

// Per-vesicle index arrays (device pointers, length M).
struct VesIndex {
  const int32_t* N;     // points of vesicle v (even, 8..NMAX)
  const int64_t* off;   // first point of v in the point arrays
  const int64_t* moff;  // first element of v's matrix scratch (MatLayout::TOTAL N^2 elements)
  const int64_t* toff;  // first double of the tables for v's N
  const int32_t* order; // CTA b of a per-vesicle launch works on vesicle order[b] (point counts descending,
                        // so the largest vesicles start first); null: vesicle b
  __device__ int vid(int b) const { return order ? order[b] : b; }
};

// Matrix scratch layout of one vesicle, in units of N^2 doubles from moff.
// Two operator slots of S (2N x 2N), T (2N x N), L (N x N) and SL (2N x 2N: in the FP32 scratch the low
// part S - S_hi of the FP64 S; unused in the FP64 scratch), then D4, B, W, A.
struct MatLayout {
  static __host__ __device__ inline int64_t slot(int s) { return s ? 11 : 0; }
  static constexpr int64_t S = 0, T = 4, L = 6, SL = 7;
  static constexpr int64_t D4 = 22, B = 23, W = 27, A = 29, TOTAL = 33;
};

// Fused multiply-add in the operands' own precision (a plain fma() on floats would promote to FP64).
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double (blockDim.x a multiple of 32, <= 1024). All threads get it.
__device__ inline double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

__device__ inline double block_max(double v, double* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = red[0];
  for (int w = 1; w < nw; ++w) t = fmax(t, red[w]);
  return t;
}

// out_i = sum_j c[(i - j) mod N] v_j : a circulant matrix-vector product (thread i).
__device__ __forceinline__ double circ_row(const double* c, const double* v, int N, int i) {
  double acc = 0.0;
  int m = i;
  for (int j = 0; j < N; ++j) {
    acc = fma(c[m], v[j], acc);
    m = (m == 0) ? N - 1 : m - 1;
  }
  return acc;
}

}  // namespace vs
