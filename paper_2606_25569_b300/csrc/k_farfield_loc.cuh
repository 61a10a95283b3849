// Local expansions for the multipole far field (VS_FLAG_FARFIELD_MULTIPOLE; the paper names the fast
// multipole method as the route to O(M) far-field cost, Sec. 4.1).
//
// A source vesicle B contributes at a target z through its order-P expansion about its centre c_B
// (k_ff_moments, mp_far): with q = z - c_B and zeta = 1/q,
//   u = -A0 log|q| + A0/2 + T1(zeta)/2 + conj(E(zeta))/2 + q conj(S_A(zeta))/2,
// T1, E, S_A power series in zeta starting at zeta^1. For a target vesicle A whose centre is far from c_B,
// put z = c_A + w and d = c_A - c_B: each series F = sum_k f_k (d + w)^-k has the Taylor expansion
//   F = sum_m L_m w^m,  L_m = (-1/d)^m sum_k C(k+m-1, m) f_k d^-k,
// and log|d + w| = log|d| + Re sum_{m>=1} (-1)^(m+1) (w/d)^m / m. Summed over the far sources, the velocity
// at every point of A is
//   u(w) = C + H(w)/2 + conj(K(w))/2 + w conj(S(w))/2
// with C = sum_B (-A0 log|d| + A0/2), H = sum_B (L[T1] - A0 l), K = sum_B (L[E] + conj(d) L[S_A] - conj(A0) l),
// S = sum_B L[S_A], l the log series: three power series of degree P per target vesicle (the translation
// that fast multipole methods call multipole-to-local). A pair (A, B) takes this route when
// |c_A - c_B| > 2 (reach_A + reach_B); the truncation error is then below about 2^-(P+1) of B's density
// scale (measured on 64-point vesicles: 5e-9 at twice, 1e-11 at three times the summed radii). The other
// source vesicles of A are listed (ascending) and summed per target point as before: B's expansion where
// the point is beyond three reach radii of c_B, the point sum with the near test inside.
#pragma once
#include "k_farfield.cuh"

namespace vs {

constexpr int FFL_LIST = 128;     // listed (not separated) source vesicles per target vesicle
constexpr float FFL_SEP2 = 4.0f;  // separated when |c_A - c_B|^2 > 4 (reach_A + reach_B)^2

// floats of one local expansion of order P: C, then H, K, S (P + 1 complex coefficients each)
__host__ __device__ constexpr int ffl_floats(int P) { return 2 + 6 * (P + 1); }

__host__ __device__ constexpr float ffl_binom(int n, int r) {
  double c = 1.0;
  for (int i = 1; i <= r; ++i) c = c * (n - r + i) / i;
  return (float)c;
}

struct FfLocArgs {
  int M;
  const float4* centre32;  // [M] centre hi/lo
  const float2* h2;        // [M] (h^2, reach^2)
  const float4* coef;      // [M][2 (P + 1)] expansion coefficients (k_ff_moments)
  const float2* a0;        // [M] total weighted density A0
  float* loc;              // [M][ffl_floats(P)]
  int* ncnt;               // [M] number of source vesicles that are not separated (may exceed FFL_LIST)
  int* nlist;              // [M][FFL_LIST] those source vesicles, ascending
};

__device__ __forceinline__ bool ffl_separated(float4 ca, float ra, float4 cb, float rb, float& dx, float& dy) {
  dx = (ca.x - cb.x) + (ca.z - cb.z);
  dy = (ca.y - cb.y) + (ca.w - cb.w);
  const float s = ra + rb;
  return fmaf(dx, dx, dy * dy) > FFL_SEP2 * s * s;
}

// Adds to acc (C, H, K, S as in ffl_floats) the local expansion about a target centre c_A of one source
// expansion (coefficients cf, total density A0) about c_B, d = (dx, dy) = c_A - c_B: the multipole-to-local
// translation written out above.
template <int P>
__device__ __forceinline__ void ffl_translate(float* acc, float dx, float dy, const float4* __restrict__ cf,
                                              float2 A0) {
  constexpr int NT = P + 1;
  constexpr int OH = 2, OK = 2 + 2 * NT, OS = 2 + 4 * NT;
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2
  const float dd = fmaf(dx, dx, dy * dy);
  const float id = 1.f / dd;
  const float zr = dx * id, zi = -dy * id;  // zeta = 1/d
  float pr[NT + 1], pi[NT + 1];             // zeta^k
  pr[0] = 1.f;
  pi[0] = 0.f;
#pragma unroll
  for (int k = 1; k <= NT; ++k) {
    pr[k] = pr[k - 1] * zr - pi[k - 1] * zi;
    pi[k] = pr[k - 1] * zi + pi[k - 1] * zr;
  }
  // constant: -A0 log|d| + A0/2
  const float ld = hl2 * fast_lg2(dd);
  acc[0] = fmaf(A0.x, ld + 0.5f, acc[0]);
  acc[1] = fmaf(A0.y, ld + 0.5f, acc[1]);
#pragma unroll
  for (int sigma = 0; sigma < 3; ++sigma) {  // T1, E, S_A
    float gr[NT + 1], gi[NT + 1];            // f_k zeta^k
#pragma unroll
    for (int k = 1; k <= NT; ++k) {
      const float4 c = cf[(k - 1) * 2 + (sigma == 1 ? 1 : 0)];
      const float fr = sigma == 2 ? c.z : c.x, fi = sigma == 2 ? c.w : c.y;
      gr[k] = fr * pr[k] - fi * pi[k];
      gi[k] = fr * pi[k] + fi * pr[k];
    }
    float mr = 1.f, mi = 0.f;  // (-zeta)^m
#pragma unroll
    for (int m = 0; m < NT; ++m) {
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int k = 1; k <= NT; ++k) {
        const float b = ffl_binom(k + m - 1, m);
        sr = fmaf(b, gr[k], sr);
        si = fmaf(b, gi[k], si);
      }
      const float lr = sr * mr - si * mi, li = sr * mi + si * mr;  // L_m
      if (sigma == 0) {  // H += L[T1] - A0 l_m, l_m = -(-zeta)^m / m
        acc[OH + 2 * m] += lr;
        acc[OH + 2 * m + 1] += li;
        if (m > 0) {
          const float im = 1.f / m;
          acc[OH + 2 * m] = fmaf(im, A0.x * mr - A0.y * mi, acc[OH + 2 * m]);
          acc[OH + 2 * m + 1] = fmaf(im, A0.x * mi + A0.y * mr, acc[OH + 2 * m + 1]);
        }
      } else if (sigma == 1) {  // K += L[E] - conj(A0) l_m
        acc[OK + 2 * m] += lr;
        acc[OK + 2 * m + 1] += li;
        if (m > 0) {
          const float im = 1.f / m;
          acc[OK + 2 * m] = fmaf(im, A0.x * mr + A0.y * mi, acc[OK + 2 * m]);
          acc[OK + 2 * m + 1] = fmaf(im, A0.x * mi - A0.y * mr, acc[OK + 2 * m + 1]);
        }
      } else {  // S += L[S_A]; K += conj(d) L[S_A]
        acc[OS + 2 * m] += lr;
        acc[OS + 2 * m + 1] += li;
        acc[OK + 2 * m] = fmaf(dx, lr, fmaf(dy, li, acc[OK + 2 * m]));
        acc[OK + 2 * m + 1] = fmaf(dx, li, fmaf(-dy, lr, acc[OK + 2 * m + 1]));
      }
      const float nr = -(mr * zr - mi * zi), ni = -(mr * zi + mi * zr);
      mr = nr;
      mi = ni;
    }
  }
}

// Sum of the CTA's partial local expansions (lanes, then warps in order), stored for target vesicle A.
template <int P>
__device__ __forceinline__ void ffl_store(const float* acc, float* __restrict__ loc) {
  constexpr int NF = ffl_floats(P);
  __shared__ float part[4][NF];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    float v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part[wid][i] = v;
  }
  __syncthreads();
  for (int i = tid; i < NF; i += 128) loc[i] = ((part[0][i] + part[1][i]) + part[2][i]) + part[3][i];
}

// Target vesicle A against every source vesicle (128 threads): thread j translates the separated source
// vesicles j, j + 128, ... into its own partial local expansion; the partials are summed across the CTA in
// a fixed order. Then the source vesicles that are not separated are listed in ascending order.
template <int P>
__device__ __forceinline__ void ffl_local_all(const FfLocArgs& a, int A) {
  constexpr int NT = P + 1, NF = ffl_floats(P);
  __shared__ int wcount[4];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const float4 ca = a.centre32[A];
  const float ra = sqrtf(a.h2[A].y);
  float acc[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) acc[i] = 0.f;
  for (int B = tid; B < a.M; B += 128) {
    float dx, dy;
    if (B == A || !ffl_separated(ca, ra, a.centre32[B], sqrtf(a.h2[B].y), dx, dy)) continue;
    ffl_translate<P>(acc, dx, dy, a.coef + (int64_t)B * 2 * NT, a.a0[B]);
  }
  ffl_store<P>(acc, a.loc + (int64_t)A * NF);
  // list of the source vesicles that are not separated, ascending
  int base = 0;
  for (int B0 = 0; B0 < a.M; B0 += 128) {
    const int B = B0 + tid;
    float dx, dy;
    const bool listed = B < a.M && B != A && !ffl_separated(ca, ra, a.centre32[B], sqrtf(a.h2[B].y), dx, dy);
    const unsigned bal = __ballot_sync(0xffffffffu, listed);
    __syncthreads();  // the previous pass's reads of wcount are over
    if (lane == 0) wcount[wid] = __popc(bal);
    __syncthreads();
    int off = base;
    for (int w2 = 0; w2 < wid; ++w2) off += wcount[w2];
    off += __popc(bal & ((1u << lane) - 1u));
    if (listed && off < FFL_LIST) a.nlist[(int64_t)A * FFL_LIST + off] = B;
    base += wcount[0] + wcount[1] + wcount[2] + wcount[3];
  }
  if (tid == 0) a.ncnt[A] = base;
}

// One CTA of 128 threads per target vesicle: ffl_local_all.
template <int P>
__global__ void __launch_bounds__(128) k_ff_local(FfLocArgs a) {
  ffl_local_all<P>(a, blockIdx.x);
}

// One CTA of 128 threads per target vesicle, a thread per target point: the local expansion of the
// separated source vesicles, then the listed ones per point (expansion beyond three reach radii, point sum
// with the near test inside; all of them in ascending order when the list overflowed), Neumaier-compensated.
template <int P>
__global__ void __launch_bounds__(128) k_farfield_loc(FarFieldArgs a, FfLocArgs l, const float4* __restrict__ src) {
  constexpr int NT = P + 1, NF = ffl_floats(P);
  constexpr int OH = 2, OK = 2 + 2 * NT, OS = 2 + 4 * NT;
  __shared__ float sl[NF];
  const int A = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < NF; i += 128) sl[i] = l.loc[(int64_t)A * NF + i];
  __syncthreads();
  const int64_t o = a.voff[A];
  const int N = (int)(a.voff[A + 1] - o);
  if (tid >= N) return;
  const int64_t t = o + tid;
  const float4 ts = src[t];
  const float4 tc = l.centre32[A];
  const float wr = ts.x, wi = ts.y;  // the target relative to its vesicle's centre
  // Horner in w for H, K, S
  float hr = 0.f, hi = 0.f, kr = 0.f, ki = 0.f, sr = 0.f, si = 0.f;
#pragma unroll
  for (int m = NT - 1; m >= 0; --m) {
    float r;
    r = hr * wr - hi * wi + sl[OH + 2 * m]; hi = hr * wi + hi * wr + sl[OH + 2 * m + 1]; hr = r;
    r = kr * wr - ki * wi + sl[OK + 2 * m]; ki = kr * wi + ki * wr + sl[OK + 2 * m + 1]; kr = r;
    r = sr * wr - si * wi + sl[OS + 2 * m]; si = sr * wi + si * wr + sl[OS + 2 * m + 1]; sr = r;
  }
  // u = C + H/2 + conj(K)/2 + w conj(S)/2
  float sx = sl[0] + 0.5f * (hr + kr + (wr * sr + wi * si));
  float sy = sl[1] + 0.5f * (hi - ki + (wi * sr - wr * si));
  float cx = 0.f, cy = 0.f;
  int ncnt = 0;
  const int cnt = l.ncnt[A];
  const bool listed = cnt <= FFL_LIST;
  const float ra = sqrtf(l.h2[A].y);
  const int nB = listed ? cnt : a.M;
  for (int i = 0; i < nB; ++i) {
    const int sv = listed ? l.nlist[(int64_t)A * FFL_LIST + i] : i;
    const float4 sc = l.centre32[sv];
    const float2 hb = l.h2[sv];
    if (!listed) {
      float dx, dy;
      if (sv == A || ffl_separated(tc, ra, sc, sqrtf(hb.y), dx, dy)) continue;
    }
    const float2 A0 = l.a0[sv];
    const float4 na = make_float4(hb.x, hb.y, A0.x, A0.y);
    float qx = ((tc.x - sc.x) + (tc.z - sc.z)) + ts.x;
    float qy = ((tc.y - sc.y) + (tc.w - sc.w)) + ts.y;
    float d2 = fmaf(qx, qx, qy * qy);
    float ux, uy;
    if (d2 > FF_MP_THETA2 * na.y) {
      mp_far<P, 1>(l.coef + (int64_t)sv * 2 * NT, na, &qx, &qy, &d2, &ux, &uy);
    } else if (!mp_points(a, src, t, sv, qx, qy, d2, na, ncnt, ux, uy)) {
      continue;
    }
    neumaier_add(sx, cx, ux);
    neumaier_add(sy, cy, uy);
  }
  a.u[2 * o + tid] += (double)sx + (double)cx;
  a.u[2 * o + N + tid] += (double)sy + (double)cy;
  if (a.near_mask) a.near_cnt[t] = ncnt < MAX_NEAR ? ncnt : MAX_NEAR;
}

}  // namespace vs
