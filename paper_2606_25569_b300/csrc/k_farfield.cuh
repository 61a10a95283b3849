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
// the special-function unit. A vesicle's densities sum to (nearly) zero, so its terms g_j log|r_j|^2 nearly
// cancel: each log argument is scaled by s = 2^-e, the power of two nearest below 1 / (|x_i - c_v|^2 +
// reach_v^2), which keeps the logarithms and the FP32 partial sums small for a distant vesicle (the scaled
// argument is near 1, where lg2 is most accurate), and e times the vesicle's density sum (summed in FP64) is
// added once per (target, source vesicle).
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

// The power of two 2^-e with S 2^-e in [1, 2) (S > 0, normal), and e: a log-argument scale whose logarithm
// is exact and whose product with |r|^2 is exact.
__device__ __forceinline__ float pow2_scale(float S, float& e) {
  const int ex = ((__float_as_int(S) >> 23) & 0xff) - 127;
  e = (float)ex;
  return __int_as_float((127 - ex) << 23);
}

// The same with e even, and t = 2^(-e/2): scaling both points of a pair by t scales |r|^2 by 2^-e exactly
// (powers of two commute with rounding), so the log argument needs no multiply of its own, while the
// Stokeslet's (r . g) r / |r|^2 does not change at all.
__device__ __forceinline__ float pow2_scale_even(float S, float& t) {
  int ex = ((__float_as_int(S) >> 23) & 0xff) - 127;
  ex -= ex & 1;  // down to even (two's complement: -3 -> -4)
  t = __int_as_float((127 - ex / 2) << 23);
  return __int_as_float((127 - ex) << 23);
}

__device__ __forceinline__ void neumaier_add(float& s, float& c, float p) {
  const float t = s + p;
  c += (fabsf(s) >= fabsf(p)) ? ((s - t) + p) : ((p - t) + s);
  s = t;
}

// Sum over the sources j0..j1-1 (shared memory) of one vesicle for the target at (qx, qy) in the
// vesicle's frame; with MIN the smallest |r|^2 is tracked too.
// The log arguments are scaled by sc (see k_farfield_f32).
template <bool MIN>
__device__ __forceinline__ void ff_sum(const float4* sh, int j0, int j1, float qx, float qy, float sc, float& ax,
                                       float& ay, float& lx, float& ly, float& mn) {
#pragma unroll 16
  for (int j = j0; j < j1; ++j) {
    const float4 s = sh[j];
    const float rx = qx - s.x, ry = qy - s.y;
    const float r2 = fmaf(rx, rx, ry * ry);
    if (MIN) mn = fminf(mn, r2);
    const float lg = fast_lg2(r2 * sc);
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
                                                          const float2* __restrict__ h2,
                                                          const float2* __restrict__ gsum) {
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
      const float q2 = fmaf(qx, qx, qy * qy);
      const bool test = a.near_mask && q2 <= nr.y;
      float le;
      const float ls = pow2_scale(q2 + nr.y, le);
      float ax = 0.f, ay = 0.f, lx = 0.f, ly = 0.f, mn = 3.0e38f;
      if (test)
        ff_sum<true>(sh, j0, j1, qx, qy, ls, ax, ay, lx, ly, mn);
      else
        ff_sum<false>(sh, j0, j1, qx, qy, ls, ax, ay, lx, ly, mn);
      if (test && mn <= nr.x) {
        if (ncnt < MAX_NEAR) a.near_v[t * MAX_NEAR + ncnt] = sv;
        else atomicOr(a.err, ERR_NEAR_OVERFLOW);
        ++ncnt;
      } else {
        const float2 gs = gsum[sv];
        neumaier_add(sx, cx, fmaf(hl2, fmaf(le, gs.x, lx), ax));
        neumaier_add(sy, cy, fmaf(hl2, fmaf(le, gs.y, ly), ay));
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

// ---- Vesicle multipole far field (FP32; opt-in). A source vesicle far from the target (|q| > 3 R_v,
// q = target - c_v, R_v the reach radius) contributes through a truncated expansion of its Stokeslet sum
// about its centre instead of its N point terms; nearer vesicles are summed point by point exactly as in
// k_farfield_f32 (near-pair test and lists included). With s_j = X_vj - c_v, g_j as above, complex numbers
// for 2-vectors and zeta = 1/q, the pair term -g log|w| + (w . g) w / |w|^2, w = q - s_j, equals
// -g log|w| + g/2 + (w / conj(w)) conj(g)/2; expanding log(1 - s/q) and 1/conj(w) in powers of s/q gives
//   u = -A_0 log|q| + A_0/2 + T1/2 + conj(E)/2 + q conj(S_A)/2,
//   T1 = sum_{k=1..P} (A_k/k) zeta^k,  S_A = sum_{k=1..P+1} A_{k-1} zeta^k,
//   E  = sum_{k=1..P+1} (conj(B_k)/k [k <= P] - conj(D_{k-1})) zeta^k,
// A_k = sum_j g_j s_j^k, B_k = sum_j g_j conj(s_j)^k, D_k = sum_j conj(g_j) s_j conj(s_j)^k (moments in FP64,
// stored in FP32). The truncation error is below (R_v/|q|)^(P+1) ~ 1/3^(P+1) of the vesicle's density scale.
constexpr int FF_MP_P = 12;            // expansion order
constexpr float FF_MP_THETA2 = 9.0f;   // far when |q|^2 > 9 R_v^2

// Moments of every vesicle: one CTA per vesicle, one thread per point; each thread forms s^k (k = 0..P+1)
// by repeated products and its terms of A_k, B_k, D_k in FP64 into shared memory (ffm_smem bytes), and one
// thread per moment component sums them in point order. coef[v][k - 1], k = 1..P+1: (A_k/k [k <= P], A_{k-1}) and
// (E_k, 0, 0) as float4 pairs; a0[v] = A_0.
inline size_t ffm_smem(int P, int threads) { return (size_t)6 * (P + 2) * threads * sizeof(double); }

// Coefficients (k = 1..P+1; thread k) and A_0 (thread 0) of an expansion from its moments A, B, D (K = P + 2
// of each), written for one vesicle or cluster: coef points at its 2 (P + 1) float4.
template <int P>
__device__ __forceinline__ void ffm_coef(int k, const double2* sA, const double2* sB, const double2* sD,
                                         float4* __restrict__ coef, float2* __restrict__ a0) {
  if (k >= 1 && k <= P + 1) {
    const double ik = 1.0 / k;
    const double2 c1 = (k <= P) ? make_double2(sA[k].x * ik, sA[k].y * ik) : make_double2(0.0, 0.0);
    const double2 cA = sA[k - 1];
    double er = -sD[k - 1].x, ei = sD[k - 1].y;  // -conj(D_{k-1})
    if (k <= P) {
      er += sB[k].x * ik;   // conj(B_k)/k
      ei -= sB[k].y * ik;
    }
    float4* c = coef + (k - 1) * 2;
    c[0] = make_float4((float)c1.x, (float)c1.y, (float)cA.x, (float)cA.y);
    c[1] = make_float4((float)er, (float)ei, 0.f, 0.f);
  }
  if (k == 0) *a0 = make_float2((float)sA[0].x, (float)sA[0].y);
}

// raw (optional): the moments themselves, [M][3 K] double2 (A_0..A_{K-1}, B_..., D_...), for the cluster tree.
template <int P>
__global__ void __launch_bounds__(NMAX) k_ff_moments(const int64_t* __restrict__ voff, const float4* __restrict__ src,
                                                     float4* __restrict__ coef, float2* __restrict__ a0,
                                                     double2* __restrict__ raw = nullptr) {
  constexpr int K = P + 2;
  extern __shared__ double mvals[];  // [6 K][blockDim]: every thread's terms, summed per moment below
  __shared__ double2 sA[K], sB[K], sD[K];
  const int v = blockIdx.x, j = threadIdx.x, nt = blockDim.x;
  const int64_t o = voff[v], n = voff[v + 1] - o;
  double sx = 0.0, sy = 0.0, gx = 0.0, gy = 0.0;
  if (j < n) {
    const float4 q = src[o + j];
    sx = q.x; sy = q.y; gx = q.z; gy = q.w;
  }
  double pr = 1.0, pi = 0.0;  // s^k
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double* t = mvals + (6 * k) * nt + j;
    t[0 * nt] = gx * pr - gy * pi;  // g s^k
    t[1 * nt] = gx * pi + gy * pr;
    t[2 * nt] = gx * pr + gy * pi;  // g conj(s)^k = g conj(s^k)
    t[3 * nt] = gy * pr - gx * pi;
    const double wr = sx * pr + sy * pi, wi = sy * pr - sx * pi;  // s conj(s^k)
    t[4 * nt] = gx * wr + gy * wi;  // conj(g) s conj(s^k)
    t[5 * nt] = gx * wi - gy * wr;
    const double nr = pr * sx - pi * sy;
    pi = pr * sy + pi * sx;
    pr = nr;
  }
  __syncthreads();
  // one thread per moment component sums the points' terms in order (FP64 adds run at a low rate on this
  // part: this takes far fewer of them than tree reductions of every term across the warp)
  for (int e = j; e < 6 * K; e += nt) {
    const double* row = mvals + (int64_t)e * nt;
    double x = 0.0;
    for (int q = 0; q < n; ++q) x += row[q];
    const int k = e / 6, c = e - 6 * k;
    reinterpret_cast<double*>((c >> 1) == 0 ? sA : (c >> 1) == 1 ? sB : sD)[2 * k + (c & 1)] = x;
  }
  __syncthreads();
  ffm_coef<P>(j, sA, sB, sD, coef + (int64_t)v * (P + 1) * 2, a0 + v);
  if (raw)
    for (int e = j; e < 3 * K; e += nt) raw[(int64_t)v * 3 * K + e] = e < K ? sA[e] : e < 2 * K ? sB[e - K] : sD[e - 2 * K];
}

// Horner evaluation of a far vesicle's expansion (its coefficients c, (h^2, reach^2, A0) in na)
// for E targets at once (q_e = (qx[e], qy[e]), |q_e|^2 = d2[e]): every coefficient load serves all E.
template <int P, int E>
__device__ __forceinline__ void mp_far(const float4* c, float4 na, const float* qx, const float* qy, const float* d2,
                                       float* ux, float* uy) {
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2
  float zr[E], zi[E], t1r[E], t1i[E], sar[E], sai[E], er[E], ei[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const float inv = fast_rcp(d2[e]);
    zr[e] = qx[e] * inv;
    zi[e] = -qy[e] * inv;  // zeta = 1/q
    t1r[e] = t1i[e] = sar[e] = sai[e] = er[e] = ei[e] = 0.f;
  }
#pragma unroll
  for (int k = P; k >= 0; --k) {  // Horner from the top coefficient (index k = power - 1)
    const float4 c0 = c[2 * k], c1 = c[2 * k + 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      float r;
      r = fmaf(t1r[e], zr[e], fmaf(-t1i[e], zi[e], c0.x)); t1i[e] = fmaf(t1r[e], zi[e], fmaf(t1i[e], zr[e], c0.y)); t1r[e] = r;
      r = fmaf(sar[e], zr[e], fmaf(-sai[e], zi[e], c0.z)); sai[e] = fmaf(sar[e], zi[e], fmaf(sai[e], zr[e], c0.w)); sar[e] = r;
      r = fmaf(er[e], zr[e], fmaf(-ei[e], zi[e], c1.x)); ei[e] = fmaf(er[e], zi[e], fmaf(ei[e], zr[e], c1.y)); er[e] = r;
    }
  }
#pragma unroll
  for (int e = 0; e < E; ++e) {
    // the series start at zeta^1: one more factor zeta
    float r;
    r = t1r[e] * zr[e] - t1i[e] * zi[e]; t1i[e] = t1r[e] * zi[e] + t1i[e] * zr[e]; t1r[e] = r;
    r = sar[e] * zr[e] - sai[e] * zi[e]; sai[e] = sar[e] * zi[e] + sai[e] * zr[e]; sar[e] = r;
    r = er[e] * zr[e] - ei[e] * zi[e]; ei[e] = er[e] * zi[e] + ei[e] * zr[e]; er[e] = r;
    const float lq = hl2 * fast_lg2(d2[e]);  // -log|q|
    // u = -A0 log|q| + A0/2 + T1/2 + conj(E)/2 + q conj(S_A)/2
    ux[e] = fmaf(na.z, lq + 0.5f, 0.5f * (t1r[e] + er[e] + (qx[e] * sar[e] + qy[e] * sai[e])));
    uy[e] = fmaf(na.w, lq + 0.5f, 0.5f * (t1i[e] - ei[e] + (qy[e] * sar[e] - qx[e] * sai[e])));
  }
}

// Point sum over vesicle sv's sources (global memory) for the target at q, with the near test when the
// target is within reach; returns false (and records sv in the target's near list) for a near pair.
__device__ __forceinline__ bool mp_points(const FarFieldArgs& a, const float4* __restrict__ src, int64_t t, int sv,
                                          float qx, float qy, float d2, float4 na, int& ncnt, float& ux, float& uy) {
  const float hl2 = -0.34657359027997264f;
  const bool test = a.near_mask && d2 <= na.y;
  float ax = 0.f, ay = 0.f, lx = 0.f, ly = 0.f, mn = 3.0e38f;
  const int64_t j0 = a.voff[sv], j1 = a.voff[sv + 1];
  for (int64_t j = j0; j < j1; ++j) {
    const float4 s = __ldg(src + j);
    const float rx = qx - s.x, ry = qy - s.y;
    const float r2 = fmaf(rx, rx, ry * ry);
    if (test) mn = fminf(mn, r2);
    const float lg = fast_lg2(r2);
    const float iv = fast_rcp(r2);
    lx = fmaf(lg, s.z, lx);
    ly = fmaf(lg, s.w, ly);
    const float q = fmaf(rx, s.z, ry * s.w) * iv;
    ax = fmaf(q, rx, ax);
    ay = fmaf(q, ry, ay);
  }
  if (test && mn <= na.x) {
    if (ncnt < MAX_NEAR) a.near_v[t * MAX_NEAR + ncnt] = sv;
    else atomicOr(a.err, ERR_NEAR_OVERFLOW);
    ++ncnt;
    return false;
  }
  ux = fmaf(hl2, lx, ax);
  uy = fmaf(hl2, ly, ay);
  return true;
}

}  // namespace vs
