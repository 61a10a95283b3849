// Symmetric evaluation of the all-pairs far-field single-layer sum (Sec. 2.2.2, Sec. 4.1, Algorithm 4).
//
// The 2D Stokeslet is even in r: G(-r) = G(r), with G(r) g = -log|r| g + (r . g) r / |r|^2. So one
// evaluation of the pair (x_i in vesicle A, X_j in vesicle B) gives both reactions: the velocity at x_i
// from the density g_j and the velocity at X_j from g_i, sharing r, |r|^2, log|r|^2 and 1/|r|^2. Every
// unordered pair of distinct vesicles is visited once, which halves the special-function work of the
// per-target kernel (k_farfield_f32) and cuts the FP32 work per ordered pair by about a third.
//
// Uneven point counts. Each vesicle is handled as R = 1, 2 or 4 segments of 32 points (its class: N <= 32,
// <= 64, <= 128). Its sources are copied into a padded array of 32 R entries (k_ffs_pad); a padding entry
// repeats the vesicle's first point with zero density, so it adds nothing as a source and changes no
// distance minimum, and what is computed for it as a target is discarded. The kernel works in the
// symmetric order, the vesicles sorted by class (4, 2, 1), cut into chunks of at most FFS_V vesicles of one
// class; a tile is a pair of chunks (I, J), I <= J, so its rows are of class R_I >= R_J of its columns, and
// each pair of classes has its own instantiation k_farfield_sym<R_I, R_J> and persistent launch.
//
// Work decomposition. A CTA stages chunk J's padded points (the columns) in shared memory and its W warps
// take the row vesicles of chunk I, one per warp. For a row vesicle A and a column vesicle B the lanes
// hold A's points (lane + 32 r) in registers; at step k = 0..31 lane l pairs them with B's points
// ((l + k) mod 32) + 32 c, read from a shared-memory copy in which each 32-point segment is stored twice
// so that the index never wraps. The row reactions accumulate in place; the column reactions accumulate
// in registers that are passed one lane down after every step, so that after 32 steps lane l holds the
// total for B's points l + 32 c. Warps visit the column vesicles in a rotated order (warp w takes column
// (w + k) mod n_J at iteration k, a barrier between iterations), so no two warps add into the same column
// accumulators at once and every accumulator receives its terms in a fixed order.
//
// Near pairs (Sec. 4.1, Algorithm 4): the minimum |r|^2 over B (for each target of A) and over A (for each
// target of B) is tracked only when the two vesicles' reach circles overlap; a target with min |r|^2 <= h^2
// of the source vesicle skips that vesicle's sum and records it in its near list. Lists are filled with
// atomics and sorted by the reduction kernel, so they equal the per-target kernel's (ascending source
// vesicle, at most MAX_NEAR; more sets ERR_NEAR_OVERFLOW).
//
// Common logarithm: the densities of a vesicle sum to (nearly) zero, so its terms g_j log|r_j|^2 nearly
// cancel. Each log argument is scaled by s = 2^-e, the power of two with even exponent at or below
// 1 / (|c_A - c_B|^2 + reach_A^2 + reach_B^2), the same for both reactions of the pair: log2(|r|^2 s) is small
// for separated vesicles, which keeps the FP32 partial sums small, and e times the source vesicle's density
// sum (summed in FP64) is added once per pair (Sum_j g_j log2|r_j|^2 = Sum_j g_j log2(|r_j|^2 s) + e Sum_j g_j;
// the scaling and e are exact). The scaling is applied to the coordinates (both points of a pair times
// 2^(-e/2)), which leaves (r . g) r / |r|^2 unchanged bit for bit and costs no operation per pair.
//
// Precision: per (target, source vesicle) partial sums in FP32 as in k_farfield_f32, added to running
// sums with Neumaier compensation (registers for the rows, shared memory for the columns). Tile (I, J)
// writes the contributions of chunk J to the points of chunk I and those of chunk I to the points of
// chunk J into slots part[J][.] and part[I][.] (each slot written exactly once, as the compensated float
// pair); k_farfield_sym_reduce adds the slots of each point in chunk order in double-float arithmetic
// (FP64 adds run at 1/64 of the FP32 rate on this part). The result is deterministic and independent of
// which CTA takes which tile; it differs from the per-target kernel's by FP32 rounding only.
#pragma once
#include "dfloat.cuh"
#include "k_farfield.cuh"

namespace vs {

#ifndef FFS_UNROLL
#define FFS_UNROLL 16
#endif
constexpr int FFS_STEPS_UNROLLED = FFS_UNROLL;  // steps of the 32-step lane rotation unrolled together

constexpr int FFS_V = 16;  // vesicles per chunk (uneven point counts; equal N: 8, 16 or 32, autotuned)
constexpr int FFS_W = 8;   // warps per CTA

struct FfSymArgs {
  int64_t P;            // real points (targets = sources)
  int M;
  int nchunk;
  int near_mask;
  float4* part;         // [slots][P]: velocity at each point from the vesicles of one chunk (x sum and
                        // compensation, y sum and compensation); chunk K writes slot K % slots
  int slots;            // nchunk (one pass), or the group size S of the phased evaluation
  int* near_cnt;        // [P], zero before each launch when near_mask
  int* near_v;          // [P * MAX_NEAR]
  unsigned* err;
  // the symmetric order: position s holds vesicle vid[s]; classes (segments R) descending
  const int* vid;       // [M]
  const int64_t* poff;  // [M] first entry of s in the padded sources (32 R_s entries each)
  const int64_t* roff;  // [M] first point of s in the point arrays
  const int* nreal;     // [M] points of s
  const int2* chunk;    // [nchunk] (first position, vesicles)
  const float4* psrc;   // padded sources (x - c_v, y - c_v, g_x, g_y)
};

// The tiles of one pair of classes and their counter.
struct FfSymTiles {
  const int2* tiles;   // [ntile] (I, J), I <= J
  int ntile;
  unsigned* ctr;       // next tile; zero before each launch
};

// Shared memory of one CTA (float4 units): the staged column chunk (64 per segment: each 32-point
// segment twice) and the column accumulators (32 per segment: sum_x, comp_x, sum_y, comp_y).
inline size_t ffs_smem_bytes(int RC, int V) { return (size_t)V * 3 * 32 * RC * sizeof(float4); }

// Segments (of 32 points) of a vesicle of N points in the symmetric kernel.
__host__ __device__ inline int ffs_segments(int N) { return N <= 32 ? 1 : N <= 64 ? 2 : 4; }

__device__ __forceinline__ void ffs_near(const FfSymArgs& a, int64_t t, int v) {
  const int slot = atomicAdd(&a.near_cnt[t], 1);
  if (slot < MAX_NEAR) a.near_v[t * MAX_NEAR + slot] = v;
  else atomicOr(a.err, ERR_NEAR_OVERFLOW);
}

// One (row vesicle A, column vesicle B) pair: row targets (tx, ty) relative to B's centre, times t, with
// their own densities rp.zw (and hl2 times them in gxs, gys); B's staged points at colB, taken times t.
// Row partial sums in lx..ay, column partial sums (log term already scaled) in ux, uy; minima of the
// scaled |r|^2 when MIN. Both points of a pair scaled by t = 2^(-e/2) put the log argument |r|^2 2^-e
// into range without a multiply (pow2_scale_even); r is taken as source minus target (the pair terms
// are even in r).
template <int RR, int RC, bool MIN>
__device__ __forceinline__ void ffs_pair(const float4* __restrict__ colB, int lane, float t, const float (&tx)[RR],
                                         const float (&ty)[RR], const float4 (&rp)[RR], const float (&gxs)[RR],
                                         const float (&gys)[RR], float (&lx)[RR], float (&ly)[RR], float (&ax)[RR],
                                         float (&ay)[RR], float (&mr)[RR], float (&ux)[RC], float (&uy)[RC],
                                         float (&mc)[RC]) {
  const int from = (lane + 1) & 31;
  const float4* base = colB + lane;
#pragma unroll FFS_STEPS_UNROLLED
  for (int k = 0; k < 32; ++k) {
    float4 s[RC];
#pragma unroll
    for (int c = 0; c < RC; ++c) s[c] = base[c * 64 + k];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int c = 0; c < RC; ++c) {
        const float rx = fmaf(s[c].x, t, -tx[r]), ry = fmaf(s[c].y, t, -ty[r]);
        const float r2 = fmaf(rx, rx, ry * ry);
        if (MIN) {
          mr[r] = fminf(mr[r], r2);
          mc[c] = fminf(mc[c], r2);
        }
        const float lg = fast_lg2(r2);
        const float inv = fast_rcp(r2);
        lx[r] = fmaf(lg, s[c].z, lx[r]);
        ly[r] = fmaf(lg, s[c].w, ly[r]);
        const float q = fmaf(rx, s[c].z, ry * s[c].w) * inv;
        ax[r] = fmaf(q, rx, ax[r]);
        ay[r] = fmaf(q, ry, ay[r]);
        ux[c] = fmaf(lg, gxs[r], ux[c]);
        uy[c] = fmaf(lg, gys[r], uy[c]);
        const float qt = fmaf(rx, rp[r].z, ry * rp[r].w) * inv;
        ux[c] = fmaf(qt, rx, ux[c]);
        uy[c] = fmaf(qt, ry, uy[c]);
      }
#pragma unroll
    for (int c = 0; c < RC; ++c) {
      ux[c] = __shfl_sync(0xffffffffu, ux[c], from);
      uy[c] = __shfl_sync(0xffffffffu, uy[c], from);
      if (MIN) mc[c] = __shfl_sync(0xffffffffu, mc[c], from);
    }
  }
}

// ffs_pair for RC even in Blackwell's two-lane FP32 instructions (add, multiply and fma of float2: two FP32
// operations in one issue slot, at the same lane rate as single ones). The one-lane form is issue-bound (the
// FP32 pipe is busy in about two issue slots of three); here the column segments 2p and 2p + 1 go through
// the same instructions as the two halves of float2 values, which halves the issue slots of the FP32 work,
// so that the FP32 pipe and the special-function unit, not the issue, become the limits. The column layout
// is paired accordingly: colB[(2p + h) 64 + k] holds point
// k mod 32 of both segments, h = 0: (x_2p, x_2p+1, y_2p, y_2p+1), h = 1: (g_x 2p, g_x 2p+1, g_y 2p, g_y 2p+1).
// Coordinates scaled by t as in ffs_pair. The row sums are kept per half and added at the end.
template <int RR, int RC, bool MIN>
__device__ __forceinline__ void ffs_pair2(const float4* __restrict__ colB, int lane, float t, const float (&tx)[RR],
                                          const float (&ty)[RR], const float4 (&rp)[RR], const float (&gxs)[RR],
                                          const float (&gys)[RR], float (&lx)[RR], float (&ly)[RR], float (&ax)[RR],
                                          float (&ay)[RR], float (&mr)[RR], float (&ux)[RC], float (&uy)[RC],
                                          float (&mc)[RC]) {
  static_assert(RC % 2 == 0, "paired columns");
  constexpr int RP = RC / 2;
  const int from = (lane + 1) & 31;
  const float4* base = colB + lane;
  float2 ntx[RR], nty[RR], rz[RR], rw[RR], gx2[RR], gy2[RR], lx2[RR], ly2[RR], ax2[RR], ay2[RR], ux2[RP], uy2[RP];
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    ntx[r] = make_float2(-tx[r], -tx[r]);
    nty[r] = make_float2(-ty[r], -ty[r]);
    rz[r] = make_float2(rp[r].z, rp[r].z);
    rw[r] = make_float2(rp[r].w, rp[r].w);
    gx2[r] = make_float2(gxs[r], gxs[r]);
    gy2[r] = make_float2(gys[r], gys[r]);
    lx2[r] = ly2[r] = ax2[r] = ay2[r] = make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int p = 0; p < RP; ++p) ux2[p] = uy2[p] = make_float2(0.f, 0.f);
  const float2 t2 = make_float2(t, t);
#pragma unroll FFS_STEPS_UNROLLED
  for (int k = 0; k < 32; ++k) {
    float2 sx[RP], sy[RP], sz[RP], sw[RP];
#pragma unroll
    for (int p = 0; p < RP; ++p) {
      const float4 q0 = base[(2 * p) * 64 + k], q1 = base[(2 * p + 1) * 64 + k];
      sx[p] = make_float2(q0.x, q0.y);
      sy[p] = make_float2(q0.z, q0.w);
      sz[p] = make_float2(q1.x, q1.y);
      sw[p] = make_float2(q1.z, q1.w);
    }
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
      for (int p = 0; p < RP; ++p) {
        const float2 rx = __ffma2_rn(sx[p], t2, ntx[r]), ry = __ffma2_rn(sy[p], t2, nty[r]);
        const float2 r2 = __ffma2_rn(rx, rx, __fmul2_rn(ry, ry));
        if (MIN) {
          mr[r] = fminf(mr[r], fminf(r2.x, r2.y));
          mc[2 * p] = fminf(mc[2 * p], r2.x);
          mc[2 * p + 1] = fminf(mc[2 * p + 1], r2.y);
        }
        const float2 lg = make_float2(fast_lg2(r2.x), fast_lg2(r2.y));
        const float2 inv = make_float2(fast_rcp(r2.x), fast_rcp(r2.y));
        lx2[r] = __ffma2_rn(lg, sz[p], lx2[r]);
        ly2[r] = __ffma2_rn(lg, sw[p], ly2[r]);
        const float2 q = __fmul2_rn(__ffma2_rn(rx, sz[p], __fmul2_rn(ry, sw[p])), inv);
        ax2[r] = __ffma2_rn(q, rx, ax2[r]);
        ay2[r] = __ffma2_rn(q, ry, ay2[r]);
        ux2[p] = __ffma2_rn(lg, gx2[r], ux2[p]);
        uy2[p] = __ffma2_rn(lg, gy2[r], uy2[p]);
        const float2 qt = __fmul2_rn(__ffma2_rn(rx, rz[r], __fmul2_rn(ry, rw[r])), inv);
        ux2[p] = __ffma2_rn(qt, rx, ux2[p]);
        uy2[p] = __ffma2_rn(qt, ry, uy2[p]);
      }
#pragma unroll
    for (int p = 0; p < RP; ++p) {
      ux2[p].x = __shfl_sync(0xffffffffu, ux2[p].x, from);
      ux2[p].y = __shfl_sync(0xffffffffu, ux2[p].y, from);
      uy2[p].x = __shfl_sync(0xffffffffu, uy2[p].x, from);
      uy2[p].y = __shfl_sync(0xffffffffu, uy2[p].y, from);
      if (MIN) {
        mc[2 * p] = __shfl_sync(0xffffffffu, mc[2 * p], from);
        mc[2 * p + 1] = __shfl_sync(0xffffffffu, mc[2 * p + 1], from);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RR; ++r) {
    lx[r] = lx2[r].x + lx2[r].y;
    ly[r] = ly2[r].x + ly2[r].y;
    ax[r] = ax2[r].x + ax2[r].y;
    ay[r] = ay2[r].x + ay2[r].y;
  }
#pragma unroll
  for (int p = 0; p < RP; ++p) {
    ux[2 * p] = ux2[p].x;
    ux[2 * p + 1] = ux2[p].y;
    uy[2 * p] = uy2[p].x;
    uy[2 * p + 1] = uy2[p].y;
  }
}

// The symmetric order's per-vesicle data; with EQ (every vesicle of 32 R points, in index order) the
// identity, computed instead of read.
template <bool EQ, int R>
struct FfsIdx {
  static __device__ __forceinline__ int vid(const FfSymArgs& a, int s) { return EQ ? s : a.vid[s]; }
  static __device__ __forceinline__ int64_t poff(const FfSymArgs& a, int s) { return EQ ? (int64_t)s * 32 * R : a.poff[s]; }
  static __device__ __forceinline__ int64_t roff(const FfSymArgs& a, int s) { return EQ ? (int64_t)s * 32 * R : a.roff[s]; }
  static __device__ __forceinline__ int nreal(const FfSymArgs& a, int s) { return EQ ? 32 * R : a.nreal[s]; }
};

// CTAs per SM the register allocation must allow (256 threads each): 3 for the one-lane pair loop of small
// classes (80 registers), else 2 (the paired loop of 2 x 2 segments needs 128 registers without spills; at
// 80 registers it spilled and ran 2% slower on the dense 2000 x 64 layout).
#define FFS_MIN_CTAS(RR, RC) (((RR) <= 2 && (RC) <= 2 && (RC) % 2 == 1) ? 3 : 2)

// Persistent: each CTA takes tiles of its pair of classes (rows of RR segments, columns of RC) from t.ctr
// until none are left. blockDim = 32 * FFS_W. EQ: all vesicles have 32 RR = 32 RC points (no padding).
// V: vesicles per chunk.
template <int RR, int RC, bool EQ, int V>
__global__ void __launch_bounds__(32 * FFS_W, FFS_MIN_CTAS(RR, RC)) k_farfield_sym(FfSymArgs a, FfSymTiles t,
                                                             const float4* __restrict__ centre32,
                                                             const float2* __restrict__ h2,
                                                             const float2* __restrict__ gsum) {
  constexpr int NC = 32 * RC;  // padded points of a column vesicle
  using IR = FfsIdx<EQ, RR>;
  using IC = FfsIdx<EQ, RC>;
  extern __shared__ float4 ffs_smem[];
  __shared__ int s_tile;
  __shared__ int s_na[FFS_W];          // each warp's row vesicle: points and first point (read after the pair
  __shared__ long long s_ao[FFS_W];    // loops, so that they hold no registers there), and its density sum
  __shared__ float2 s_hga[FFS_W];      // times -ln(2)/2
  float4* col = ffs_smem;               // [V][RC][64]
  float4* acc = ffs_smem + V * 2 * NC;  // [V][NC]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2: -log|r| = hl2 log2|r|^2
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(t.ctr, 1u);
    __syncthreads();
    const int ti = s_tile;
    if (ti >= t.ntile) break;
    const int2 tij = t.tiles[ti];
    const int I = tij.x, J = tij.y;
    const int2 cI = a.chunk[I], cJ = a.chunk[J];
    const int nI = cI.y, nJ = cJ.y;
    const bool diag = I == J;
    for (int e = threadIdx.x; e < nJ * 2 * NC; e += blockDim.x) {
      const int b = e / (2 * NC), rem = e - b * 2 * NC;
      if constexpr (RC % 2 == 0) {  // paired segments (ffs_pair2)
        const int blk = rem >> 6;
        const int64_t o = IC::poff(a, cJ.x + b) + 64 * (blk >> 1) + (rem & 31);
        const float4 s0 = a.psrc[o], s1 = a.psrc[o + 32];
        col[e] = (blk & 1) ? make_float4(s0.z, s1.z, s0.w, s1.w) : make_float4(s0.x, s1.x, s0.y, s1.y);
      } else {
        col[e] = a.psrc[IC::poff(a, cJ.x + b) + 32 * (rem >> 6) + (rem & 31)];
      }
    }
    for (int e = threadIdx.x; e < nJ * NC; e += blockDim.x) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const bool rot = nJ >= FFS_W;
    const int K = rot ? nJ : nJ + FFS_W - 1;
    for (int r0 = 0; r0 < nI; r0 += FFS_W) {
      const int ai = r0 + w;
      const bool arow = ai < nI;
      const int as = cI.x + ai;
      int av = 0;
      float4 rp[RR];
      float gxs[RR], gys[RR], sxr[RR], cxr[RR], syr[RR], cyr[RR];
      float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 ha = make_float2(0.f, 0.f);
      if (arow) {
        av = IR::vid(a, as);
        if (lane == 0) {
          const float2 ga = gsum[av];
          s_na[w] = IR::nreal(a, as);
          s_ao[w] = IR::roff(a, as);
          s_hga[w] = make_float2(hl2 * ga.x, hl2 * ga.y);
        }
        ca = centre32[av];
        ha = h2[av];
      }
#pragma unroll
      for (int r = 0; r < RR; ++r) {
        rp[r] = arow ? a.psrc[IR::poff(a, as) + lane + 32 * r] : make_float4(0.f, 0.f, 0.f, 0.f);
        gxs[r] = hl2 * rp[r].z;
        gys[r] = hl2 * rp[r].w;
        sxr[r] = cxr[r] = syr[r] = cyr[r] = 0.f;
      }
      const float reach_a = sqrtf(ha.y);
      for (int k = 0; k < K; ++k) {
        int bj = rot ? w + k : k - w;
        if (rot && bj >= nJ) bj -= nJ;
        if (arow && bj >= 0 && bj < nJ && (!diag || bj > ai)) {
          const int bs = cJ.x + bj;
          const int bv = IC::vid(a, bs);
          const float4 cb = centre32[bv];
          const float2 hb = h2[bv];
          const float dx = (ca.x - cb.x) + (ca.z - cb.z), dy = (ca.y - cb.y) + (ca.w - cb.w);
          // log-argument scale of the pair (its exponent is read back after the pair loop, so that it holds no
          // register there)
          float tsc;
          const float sc = pow2_scale_even(fmaf(dx, dx, dy * dy) + (ha.y + hb.y), tsc);
          float tx[RR], ty[RR], lx[RR], ly[RR], ax[RR], ay[RR], mr[RR], ux[RC], uy[RC], mc[RC];
#pragma unroll
          for (int r = 0; r < RR; ++r) {
            tx[r] = (dx + rp[r].x) * tsc;
            ty[r] = (dy + rp[r].y) * tsc;
            lx[r] = ly[r] = ax[r] = ay[r] = 0.f;
            mr[r] = 3.0e38f;
          }
#pragma unroll
          for (int c = 0; c < RC; ++c) {
            ux[c] = uy[c] = 0.f;
            mc[c] = 3.0e38f;
          }
          // the minima are needed only when the reach circles of A and B overlap
          const float rs = reach_a + sqrtf(hb.y);
          const bool test = a.near_mask && fmaf(dx, dx, dy * dy) <= rs * rs;
          const float4* colB = col + bj * 2 * NC;
          if constexpr (RC % 2 == 0) {
            if (test)
              ffs_pair2<RR, RC, true>(colB, lane, tsc, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
            else
              ffs_pair2<RR, RC, false>(colB, lane, tsc, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
          } else {
            if (test)
              ffs_pair<RR, RC, true>(colB, lane, tsc, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
            else
              ffs_pair<RR, RC, false>(colB, lane, tsc, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
          }
          const float lsc = (float)(127 - ((__float_as_int(sc) >> 23) & 0xff));  // sc = 2^-lsc
          const float2 gb = gsum[bv];
          __syncwarp();
          const int na = EQ ? 32 * RR : s_na[w];
          const int64_t ao = s_ao[w];
#pragma unroll
          for (int r = 0; r < RR; ++r) {  // targets of A, source vesicle B
            if (!EQ && lane + 32 * r >= na) continue;
            if (test && mr[r] <= hb.x * sc) {  // minima of the scaled |r|^2
              ffs_near(a, ao + lane + 32 * r, bv);
            } else {
              neumaier_add(sxr[r], cxr[r], fmaf(hl2, fmaf(lsc, gb.x, lx[r]), ax[r]));
              neumaier_add(syr[r], cyr[r], fmaf(hl2, fmaf(lsc, gb.y, ly[r]), ay[r]));
            }
          }
          const int nb = IC::nreal(a, bs);
          const float2 hga = s_hga[w];
#pragma unroll
          for (int c = 0; c < RC; ++c) {  // targets of B, source vesicle A
            if (!EQ && lane + 32 * c >= nb) continue;
            if (test && mc[c] <= ha.x * sc) {
              ffs_near(a, IC::roff(a, bs) + lane + 32 * c, av);
            } else {
              float4& v = acc[bj * NC + lane + 32 * c];
              float4 s = v;
              neumaier_add(s.x, s.y, fmaf(lsc, hga.x, ux[c]));
              neumaier_add(s.z, s.w, fmaf(lsc, hga.y, uy[c]));
              v = s;
            }
          }
        }
        __syncthreads();
      }
      if (arow) {
        if (diag) {  // chunk I = J (so RR = RC): the row sums join the column accumulators of A's points
#pragma unroll
          for (int r = 0; r < RR; ++r) {
            float4& v = acc[ai * NC + lane + 32 * r];
            float4 s = v;
            neumaier_add(s.x, s.y, sxr[r]);
            s.y += cxr[r];
            neumaier_add(s.z, s.w, syr[r]);
            s.w += cyr[r];
            v = s;
          }
        } else {
          __syncwarp();
          const int na = EQ ? 32 * RR : s_na[w];
          const int64_t ao = s_ao[w];
#pragma unroll
          for (int r = 0; r < RR; ++r)
            if (EQ || lane + 32 * r < na)
              a.part[(int64_t)(J % a.slots) * a.P + ao + lane + 32 * r] = make_float4(sxr[r], cxr[r], syr[r], cyr[r]);
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < nJ * NC; e += blockDim.x) {  // chunk I's contributions to chunk J's points
      const int b = e / NC, i = e - b * NC;
      if (i < IC::nreal(a, cJ.x + b)) a.part[(int64_t)(I % a.slots) * a.P + IC::roff(a, cJ.x + b) + i] = acc[e];
    }
    __syncthreads();
  }
}

// Padded sources in the symmetric order: vesicle vid[s] into 32 R_s entries from poff[s], the entries past
// its N points a copy of its first point with zero density. One CTA per vesicle.
__global__ void __launch_bounds__(128) k_ffs_pad(FfSymArgs a, const float4* __restrict__ src, float4* __restrict__ psrc) {
  const int s = blockIdx.x;
  const int n = a.nreal[s], np = 32 * ffs_segments(n);
  const int64_t o = a.roff[s];
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    float4 v = src[o + (i < n ? i : 0)];
    if (i >= n) v.z = v.w = 0.f;
    psrc[a.poff[s] + i] = v;
  }
}

// u (CSR blocks [u_x(N), u_y(N)] per vesicle) += sum over chunks of part, in chunk order (double-float); near
// counts clamped to MAX_NEAR and each near list sorted ascending.
__global__ void __launch_bounds__(256) k_farfield_sym_reduce(FfSymArgs a, const int32_t* __restrict__ owner,
                                                             const int64_t* __restrict__ voff, double* __restrict__ u) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  float2 ax = make_float2(0.f, 0.f), ay = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int K = 0; K < a.nchunk; ++K) {
    const float4 v = a.part[(int64_t)K * a.P + p];
    ax = df_add(ax, make_float2(v.x, v.y));
    ay = df_add(ay, make_float2(v.z, v.w));
  }
  const double sx = (double)ax.x + (double)ax.y, sy = (double)ay.x + (double)ay.y;
  const int v = owner[p];
  const int64_t to = voff[v];
  const int64_t n = voff[v + 1] - to;
  const int64_t loc = p - to;
  u[2 * to + loc] += sx;
  u[2 * to + n + loc] += sy;
  if (a.near_mask) {
    const int c = min(a.near_cnt[p], MAX_NEAR);
    int* lst = a.near_v + p * MAX_NEAR;
    for (int i = 1; i < c; ++i) {
      const int x = lst[i];
      int j = i - 1;
      while (j >= 0 && lst[j] > x) {
        lst[j + 1] = lst[j];
        --j;
      }
      lst[j + 1] = x;
    }
    a.near_cnt[p] = c;
  }
}

// Phased evaluation (partial-sum memory bounded by S slots per point instead of one per chunk): the chunks form
// groups of S consecutive chunks, and phase (g_a, g_b), g_a <= g_b, runs the tiles (I, J) with I in g_a and J in
// g_b. In it a point of group g_a receives from the chunks of g_b only (slot J % S, each written once) and a
// point of g_b from those of g_a, so one set of S slots serves the phase; this kernel then adds the phase's
// slots of those points to u in slot order (double-float, as k_farfield_sym_reduce), the phases in a fixed
// order, so the result is deterministic. pchunk: the chunk of each point; n_a, n_b: chunks in g_a and g_b.
__global__ void __launch_bounds__(256) k_ffs_reduce_phase(FfSymArgs a, const int32_t* __restrict__ owner,
                                                          const int64_t* __restrict__ voff,
                                                          const int* __restrict__ pchunk, int ga, int gb, int na,
                                                          int nb, double* __restrict__ u) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int g = pchunk[p] / a.slots;
  if (g != ga && g != gb) return;
  const int n = (g == ga) ? nb : na;  // the slots written for this point: the chunks of the other group
  float2 ax = make_float2(0.f, 0.f), ay = make_float2(0.f, 0.f);
  for (int K = 0; K < n; ++K) {
    const float4 v = a.part[(int64_t)K * a.P + p];
    ax = df_add(ax, make_float2(v.x, v.y));
    ay = df_add(ay, make_float2(v.z, v.w));
  }
  const int v = owner[p];
  const int64_t to = voff[v];
  const int64_t nv = voff[v + 1] - to;
  const int64_t loc = p - to;
  u[2 * to + loc] += (double)ax.x + (double)ax.y;
  u[2 * to + nv + loc] += (double)ay.x + (double)ay.y;
}

// After the last phase: near counts clamped to MAX_NEAR and each near list sorted ascending (as in
// k_farfield_sym_reduce).
__global__ void __launch_bounds__(256) k_ffs_near_sort(FfSymArgs a) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.P) return;
  const int c = min(a.near_cnt[p], MAX_NEAR);
  int* lst = a.near_v + p * MAX_NEAR;
  for (int i = 1; i < c; ++i) {
    const int x = lst[i];
    int j = i - 1;
    while (j >= 0 && lst[j] > x) {
      lst[j + 1] = lst[j];
      --j;
    }
    lst[j + 1] = x;
  }
  a.near_cnt[p] = c;
}

}  // namespace vs
