// Double-float arithmetic for the mixed-precision kernels (FP64 runs at 1/64 of the FP32 rate on
// this part).
#pragma once
#include <cuda_runtime.h>

namespace vs {

// A double-float value is the unevaluated sum x + y of two floats with |y| <= ulp(x)/2
// (about 48 significant bits). Error-free transformations: TwoSum (Knuth), Fast2Sum (Dekker), the exact
// product error by FMA; dot products follow the compensated scheme Dot2 of Ogita, Rump and Oishi (2005),
// extended by the cross terms of double-float operands and folded into a double-float total every
// DF_CHUNK terms. The _rn intrinsics keep the compiler from contracting the transformations into FMAs.
constexpr int DF_CHUNK = 8;

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_of(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = two_sum(a.x, b.x);
  return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}

// Compensated accumulator: s the running FP32 sum, c the sum of its rounding errors and of the
// low-order product terms.
struct Dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float t = __fadd_rn(s, p), z = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)), e));
    s = t;
  }
  __device__ __forceinline__ void merge(float s2, float c2) {
    const float2 t = two_sum(s, s2);
    s = t.x;
    c = __fadd_rn(c, __fadd_rn(c2, t.y));
  }
  __device__ __forceinline__ float2 value() const { return two_sum(s, c); }
};


// sqrt(a) in double-float (a.x > 0 and normal): the FP32 root y0 = sqrt(a.x) plus one Newton correction
// (a - y0^2) / (2 y0) whose residual is formed exactly (y0^2 = p + e by the FMA, a.x - p exact as the two are
// within a factor of two) and summed with a.y in FP32 (Karp and Markstein, ACM TOMS 23, 1997); about 47 bits.
__device__ __forceinline__ float2 df_sqrt(float2 a) {
  const float y0 = __fsqrt_rn(a.x);
  const float p = __fmul_rn(y0, y0), e = fmaf(y0, y0, -p);
  const float r = __fsub_rn(__fadd_rn(__fsub_rn(a.x, p), a.y), e);
  return fast_two_sum(y0, __fmul_rn(r, __fmul_rn(0.5f, __frcp_rn(y0))));
}

// 1/a in double-float: the FP32 reciprocal refined by one Newton step carried out in double-float
__device__ __forceinline__ float2 df_rcp(float2 a) {
  const float2 y0 = make_float2(__frcp_rn(a.x), 0.f);
  const float2 p = df_mul(a, y0);
  const float2 e = df_add(make_float2(1.f, 0.f), make_float2(-p.x, -p.y));
  return df_add(y0, df_mul(y0, e));
}

// out_i = sum_j d[(i - j) mod N] v_j in double-float (d and v in shared memory); the compensated
// partial sums are folded into a double-float total every DF_CHUNK terms (the last chunk may be short)
__device__ __forceinline__ float2 circ_df(const float2* d, const float2* v, int N, int i) {
  float2 tot = make_float2(0.f, 0.f);
  int m = i;
  for (int j0 = 0; j0 < N; j0 += DF_CHUNK) {
    Dot2 a;
    const int j1 = min(j0 + DF_CHUNK, N);
    for (int j = j0; j < j1; ++j) {
      a.add(d[m], v[j]);
      m = (m == 0) ? N - 1 : m - 1;
    }
    tot = df_add(tot, a.value());
  }
  return tot;
}

constexpr int LOG_TAB = 512;

// Natural logarithm of a double-float x = (hi, lo) > 0 with a normal hi, table-driven (Tang, ACM TOMS 16,
// 1990): x = 2^e (m_hi + m_lo) with m_hi in [1, 2) the scaled hi, c = 1 + (k + 1/2)/LOG_TAB for k the top
// 9 fraction bits of m_hi, log x = e ln 2 + log c + log1p(f) with f = (m - c)/c in double-float
// (|f| <= 2^-10) and log1p(f) = f - f^2/2 + f^3 (1/3 - f/4 + f^2/5): the cubic part is below 2^-30, so
// plain FP32 carries it, and the next term is below 2^-62. ltd[k] = (log c hi, log c lo, 1/c hi,
// 1/c lo) is built on the host. About 47 significant bits.
__device__ __forceinline__ float2 log_df(float2 x, const float4* ltd) {
  const unsigned b = __float_as_uint(x.x);
  const int e = (int)((b >> 23) & 255u) - 127;
  const int k = (int)((b >> 14) & (unsigned)(LOG_TAB - 1));
  const float mh = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
  const float ml = ldexpf(x.y, -e);
  const float c = 1.0f + (k + 0.5f) / LOG_TAB;  // exact: 10 fraction bits
  const float4 t = ltd[k];
  const float2 f = df_mul(two_sum(__fsub_rn(mh, c), ml), make_float2(t.z, t.w));  // mh - c is exact
  const float fx = f.x;
  const float cubic = fx * fx * fx * fmaf(fx, fmaf(fx, 0.2f, -0.25f), 1.0f / 3.0f);
  const float2 f2 = df_mul(f, f);
  const float2 l1 = df_add(f, two_sum(-0.5f * f2.x, fmaf(-0.5f, f2.y, cubic)));
  constexpr float LN2_H = (float)0.69314718055994530942, LN2_L = (float)(0.69314718055994530942 - (double)LN2_H);
  const float2 eln2 = df_mul(make_float2((float)e, 0.f), make_float2(LN2_H, LN2_L));
  return df_add(df_add(eln2, make_float2(t.x, t.y)), l1);
}

}  // namespace vs
