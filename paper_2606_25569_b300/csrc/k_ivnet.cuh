// IVNet (Sec. 3.4.2, Fig. fig:net) on the tensor cores: every circular 1D convolution is a GEMM of its
// gathered input columns (BF16, K = C_in k padded to a multiple of 16) with the weights, on k_gemm_bf16
// (tcgen05, FP32 accumulation in tensor memory, bias and ReLU in the epilogue); the input gradient is the
// GEMM of the output gradient with the weights followed by the adjoint gather, the weight gradient the GEMM
// of the transposed output gradient with the transposed columns. Signals are (sample, position, channel)
// row-major FP32, rows b n + p; the batch is padded to a multiple of 128 with zero samples.
//
// Kernels (grid-stride over their elements):
//   k_iv_rows_in    network input rows [s_0(N), s_1(N), ...] (per-feature input map in FP32) -> signal (N, nch)
//   k_iv_gather     columns col[(b n_out + p) Kp + c k + t] = bf16(x[b, (s p + d (t - (k-1)/2)) mod n_in, c]);
//                   k_iv_gatherT their transpose (K-major over the rows, for the weight gradient)
//   k_iv_scatter    adjoint of the gather: dx[b, q, c] += sum over (p, t) reaching q of dcol[b n_out + p, c k + t]
//   k_iv_up         periodic linear interpolation by 2 along positions plus the finer level's signal (the
//                   prolongated coarse correction of the V-cycle); k_iv_up_T the interpolation's adjoint (added)
//   k_iv_splitsum   the weight gradient from the split-K GEMM's partial products, in order
//   k_iv_add        y = a + b (the residual stream)
//   k_iv_rows_out   projection output (channels 0, 1 of a 16-channel signal) -> rows [x(N), y(N)], with the
//                   output map when given; k_iv_rows_grad the loss gradient rows -> that signal's gradient
//   k_iv_grad       an output gradient (a channel slice of an FP32 signal gradient), masked by ReLU' from
//                   the post-activation, to FP32 (for the bias), BF16 and BF16 transposed (the GEMM operands)
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace vs {

__global__ void k_iv_rows_in(const float* __restrict__ x, int batch, int Bp, int N, int nch,
                             const float* __restrict__ shift, const float* __restrict__ scale,
                             float* __restrict__ sig) {
  const int64_t n = (int64_t)Bp * N * nch;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % nch);
    const int64_t r = e / nch;
    const int b = (int)(r / N), p = (int)(r - (int64_t)b * N);
    float v = 0.f;
    if (b < batch) {
      const int f = c * N + p;
      v = x[(int64_t)b * nch * N + f];
      if (shift) v = __fmul_rn(__fsub_rn(v, shift[f]), scale[f]);
    }
    sig[e] = v;
  }
}

struct IvConv {
  int cin, cout, k, s, d;
  int kp, coutp;  // padded K (multiple of 16) and output channels (at least 16)
};

// the gathered input of column j of row m (M = Bp n_out rows; zero in the padding columns)
__device__ __forceinline__ float iv_col(const float* __restrict__ x, int ldx, int n_in, int n_out, const IvConv& cv,
                                        int m, int j) {
  if (j >= cv.cin * cv.k) return 0.f;
  const int c = j / cv.k, t = j - c * cv.k;
  const int b = m / n_out, p = m - b * n_out;
  int q = (cv.s * p + cv.d * (t - (cv.k - 1) / 2)) % n_in;
  if (q < 0) q += n_in;
  return x[((int64_t)b * n_in + q) * ldx + c];
}

// col (M x kp, row-major); 32-bit indices (M kp < 2^31, checked at create)
__global__ void k_iv_gather(const float* __restrict__ x, int ldx, int Bp, int n_in, IvConv cv,
                            __nv_bfloat16* __restrict__ col) {
  const int n_out = n_in / cv.s;
  const int n = Bp * n_out * cv.kp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int m = e / cv.kp;
    col[e] = __float2bfloat16_rn(iv_col(x, ldx, n_in, n_out, cv, m, e - m * cv.kp));
  }
}

// colT (kp x M): the columns K-major over the rows (the weight gradient's operand), written in order
__global__ void k_iv_gatherT(const float* __restrict__ x, int ldx, int Bp, int n_in, IvConv cv,
                             __nv_bfloat16* __restrict__ colT) {
  const int n_out = n_in / cv.s;
  const int M = Bp * n_out;
  const int n = M * cv.kp;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int j = e / M;
    colT[e] = __float2bfloat16_rn(iv_col(x, ldx, n_in, n_out, cv, e - j * M, j));
  }
}

// dx (n_in positions, ldx) += the adjoint gather of dcol (M x kp)
__global__ void k_iv_scatter(const float* __restrict__ dcol, int Bp, int n_in, IvConv cv, float* __restrict__ dx,
                             int64_t ldx) {
  const int n_out = n_in / cv.s;
  const int64_t n = (int64_t)Bp * n_in * cv.cin;
  const int half = (cv.k - 1) / 2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % cv.cin);
    const int64_t r = e / cv.cin;
    const int b = (int)(r / n_in), q = (int)(r - (int64_t)b * n_in);
    float acc = 0.f;
    for (int t = 0; t < cv.k; ++t) {
      int u = (q - cv.d * (t - half)) % n_in;
      if (u < 0) u += n_in;
      if (u % cv.s) continue;
      const int p = u / cv.s;
      acc += dcol[((int64_t)b * n_out + p) * cv.kp + c * cv.k + t];
    }
    dx[r * ldx + c] += acc;
  }
}

// y (2n positions) = up(x) (n positions) + skip (2n positions, or null), C channels, contiguous
__global__ void k_iv_up(const float* __restrict__ x, const float* __restrict__ skip, int Bp, int n, int C,
                        float* __restrict__ y) {
  const int64_t total = (int64_t)Bp * 2 * n * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t r = e / C;
    const int b = (int)(r / (2 * n)), p = (int)(r - (int64_t)b * 2 * n);
    const int q = p >> 1;
    const float a = x[((int64_t)b * n + q) * C + c];
    float v = a;
    if (p & 1) v = 0.5f * (a + x[((int64_t)b * n + (q + 1 == n ? 0 : q + 1)) * C + c]);
    y[e] = skip ? v + skip[e] : v;
  }
}

// dx (n positions) += up^T(dy) (2n positions)
__global__ void k_iv_up_T(const float* __restrict__ dy, int Bp, int n, int C, float* __restrict__ dx) {
  const int64_t total = (int64_t)Bp * n * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int64_t r = e / C;
    const int b = (int)(r / n), q = (int)(r - (int64_t)b * n);
    const int64_t base = (int64_t)b * 2 * n;
    const int pm = (q == 0) ? 2 * n - 1 : 2 * q - 1;
    dx[e] += dy[(base + 2 * q) * C + c] + 0.5f * dy[(base + 2 * q + 1) * C + c] + 0.5f * dy[(base + pm) * C + c];
  }
}

__global__ void k_iv_splitsum(const float* __restrict__ part, int S, int64_t n, float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < S; ++z) s += part[(int64_t)z * n + e];
    out[e] = s;
  }
}

__global__ void k_iv_add(const float* __restrict__ a, const float* __restrict__ b, int64_t n, float* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = a[e] + b[e];
}

// rows[b][c N + p] = sig[(b N + p) 16 + c] (c = 0, 1), mapped by oscale, oshift when given
__global__ void k_iv_rows_out(const float* __restrict__ sig, int batch, int N, const float* __restrict__ oscale,
                              const float* __restrict__ oshift, float* __restrict__ rows) {
  const int64_t n = (int64_t)batch * 2 * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / (2 * N)), f = (int)(e - (int64_t)b * 2 * N);
    const int c = f / N, p = f - c * N;
    float v = sig[((int64_t)b * N + p) * 16 + c];
    if (oscale) v = fmaf(v, oscale[f], oshift[f]);
    rows[e] = v;
  }
}

// the gradient of the projection's 16-channel output from the loss gradient rows (channels >= 2 zero)
__global__ void k_iv_rows_grad(const float* __restrict__ g, int Bp, int N, float* __restrict__ sig) {
  const int64_t n = (int64_t)Bp * N * 16;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e & 15);
    const int64_t r = e >> 4;
    const int b = (int)(r / N), p = (int)(r - (int64_t)b * N);
    sig[e] = c < 2 ? g[(int64_t)b * 2 * N + c * N + p] : 0.f;
  }
}

// g (M rows, channels [0, C) of a signal with leading dimension ldg) times (post > 0) when post is non-null
// (same layout) -> gm (M x C, FP32), gb (M x C, BF16), gbT (C x M, BF16)
__global__ void k_iv_grad(const float* __restrict__ g, int64_t ldg, const float* __restrict__ post, int64_t M, int C,
                          float* __restrict__ gm, __nv_bfloat16* __restrict__ gb, __nv_bfloat16* __restrict__ gbT) {
  const int64_t n = M * C;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = e / C;
    const int c = (int)(e - m * C);
    float v = g[m * ldg + c];
    if (post && !(post[m * ldg + c] > 0.f)) v = 0.f;
    gm[e] = v;
    const __nv_bfloat16 bv = __float2bfloat16_rn(v);
    gb[e] = bv;
    gbT[(int64_t)c * M + m] = bv;
  }
}

// Samples of the signals whose Fourier features (modes <= K: a_0..a_K, b_1..b_K of x, then of y; the
// relaxation network's feature rows, row stride ld) are given: out rows [x(N), y(N)]
__global__ void k_feature_points(const float* __restrict__ feat, int rows, int64_t ld, int N, int K,
                                 float* __restrict__ out) {
  const int64_t n = (int64_t)rows * 2 * N;
  const int per = 2 * K + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / (2 * N)), f = (int)(e - (int64_t)r * 2 * N);
    const int c = f / N, p = f - c * N;
    const float* F = feat + (int64_t)r * ld + c * per;
    double v = F[0];
    for (int k = 1; k <= K; ++k) {
      double sn, cs;
      sincospi(2.0 * k * p / N, &sn, &cs);
      v += 2.0 * ((double)F[k] * cs - (double)F[K + k] * sn);
    }
    out[e] = (float)v;
  }
}

}  // namespace vs
