// Symmetric evaluation of the all-pairs far-field single-layer sum (Sec. 2.2.2, Sec. 4.1, Algorithm 4)
// for suspensions whose vesicles all have N = 32 R points.
//
// The 2D Stokeslet is even in r: G(-r) = G(r), with G(r) g = -log|r| g + (r . g) r / |r|^2. So one
// evaluation of the pair (x_i in vesicle A, X_j in vesicle B) gives both reactions: the velocity at x_i
// from the density g_j and the velocity at X_j from g_i, sharing r, |r|^2, log|r|^2 and 1/|r|^2. Every
// unordered pair of distinct vesicles is visited once, which halves the special-function work of the
// per-target kernel (k_farfield_f32) and cuts the FP32 work per ordered pair by about a third.
//
// Work decomposition. Vesicles are grouped in chunks of FFS_V; a tile is a pair of chunks (I, J), I <= J.
// A CTA stages chunk J's points (the columns) in shared memory and its W warps take the row vesicles of
// chunk I, one per warp. For a row vesicle A and a column vesicle B the lanes hold A's points
// (lane + 32 r) in registers; at step k = 0..31 lane l pairs them with B's points ((l + k) mod 32) + 32 c,
// read from a shared-memory copy in which each 32-point segment is stored twice so that the index never
// wraps. The row reactions accumulate in place; the column reactions accumulate in registers that are
// passed one lane down after every step, so that after 32 steps lane l holds the total for B's points
// l + 32 c. Warps visit the column vesicles in a rotated order (warp w takes column (w + k) mod n_J at
// iteration k, a barrier between iterations), so no two warps add into the same column accumulators at
// once and every accumulator receives its terms in a fixed order.
//
// Near pairs (Sec. 4.1, Algorithm 4): the minimum |r|^2 over B (for each target of A) and over A (for each
// target of B) is tracked only when the two vesicles' reach circles overlap; a target with min |r|^2 <= h^2
// of the source vesicle skips that vesicle's sum and records it in its near list. Lists are filled with
// atomics and sorted by the reduction kernel, so they equal the per-target kernel's (ascending source
// vesicle, at most MAX_NEAR; more sets ERR_NEAR_OVERFLOW).
//
// Precision: per (target, source vesicle) partial sums in FP32 as in k_farfield_f32, added to running
// sums with Neumaier compensation (registers for the rows, shared memory for the columns). Tile (I, J)
// writes the contributions of chunk J to the points of chunk I and those of chunk I to the points of
// chunk J into slots part[J][.] and part[I][.] (each slot written exactly once, as the compensated float
// pair); k_farfield_sym_reduce adds the slots of each point in chunk order in double-float arithmetic
// (FP64 adds run at 1/64 of the FP32 rate on this part).
// The result is deterministic and independent of which CTA takes which tile; it differs from the
// per-target kernel's by FP32 rounding only.
#pragma once
#include "dfloat.cuh"
#include "k_farfield.cuh"

namespace vs {

#ifndef FFS_UNROLL
#define FFS_UNROLL 16
#endif
constexpr int FFS_STEPS_UNROLLED = FFS_UNROLL;  // steps of the 32-step lane rotation unrolled together

constexpr int FFS_V = 16;  // vesicles per chunk
constexpr int FFS_W = 8;   // warps per CTA

struct FfSymArgs {
  int64_t P;           // points (targets = sources)
  int M, N;            // vesicles, points per vesicle (all equal)
  int nchunk, ntile;
  const int2* tiles;   // [ntile] (I, J), I <= J
  unsigned* tile_ctr;  // next tile; zero before each launch
  int near_mask;
  float4* part;        // [nchunk][P]: velocity at each point from the vesicles of one chunk (x sum and
                       // compensation, y sum and compensation)
  int* near_cnt;       // [P], zero before each launch when near_mask
  int* near_v;         // [P * MAX_NEAR]
  unsigned* err;
};

// Shared memory of one CTA (float4 units): the staged column chunk (2N per vesicle) and the
// column accumulators (N per vesicle: sum_x, comp_x, sum_y, comp_y).
inline size_t ffs_smem_bytes(int N) { return (size_t)FFS_V * 3 * N * sizeof(float4); }

__device__ __forceinline__ void ffs_near(const FfSymArgs& a, int64_t t, int v) {
  const int slot = atomicAdd(&a.near_cnt[t], 1);
  if (slot < MAX_NEAR) a.near_v[t * MAX_NEAR + slot] = v;
  else atomicOr(a.err, ERR_NEAR_OVERFLOW);
}

// One (row vesicle A, column vesicle B) pair: row targets (tx, ty) relative to B's centre with their own
// densities rp.zw (and hl2 times them in gxs, gys); B's staged points at colB. Row partial sums in
// lx..ay, column partial sums (log term already scaled) in ux, uy; minima when MIN.
template <int R, bool MIN>
__device__ __forceinline__ void ffs_pair(const float4* __restrict__ colB, int lane, const float (&tx)[R],
                                         const float (&ty)[R], const float4 (&rp)[R], const float (&gxs)[R],
                                         const float (&gys)[R], float (&lx)[R], float (&ly)[R], float (&ax)[R],
                                         float (&ay)[R], float (&mr)[R], float (&ux)[R], float (&uy)[R],
                                         float (&mc)[R]) {
  const int from = (lane + 1) & 31;
  const float4* base = colB + lane;
#pragma unroll FFS_STEPS_UNROLLED
  for (int k = 0; k < 32; ++k) {
    float4 s[R];
#pragma unroll
    for (int c = 0; c < R; ++c) s[c] = base[c * 64 + k];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) {
        const float rx = tx[r] - s[c].x, ry = ty[r] - s[c].y;
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
    for (int c = 0; c < R; ++c) {
      ux[c] = __shfl_sync(0xffffffffu, ux[c], from);
      uy[c] = __shfl_sync(0xffffffffu, uy[c], from);
      if (MIN) mc[c] = __shfl_sync(0xffffffffu, mc[c], from);
    }
  }
}

// Persistent: each CTA takes tiles from a.tile_ctr until none are left. blockDim = 32 * FFS_W.
template <int R>
__global__ void __launch_bounds__(32 * FFS_W) k_farfield_sym(FfSymArgs a, const float4* __restrict__ src,
                                                             const float4* __restrict__ centre32,
                                                             const float2* __restrict__ h2) {
  constexpr int N = 32 * R;
  extern __shared__ float4 ffs_smem[];
  __shared__ int s_tile;
  float4* col = ffs_smem;                  // [FFS_V][R][64]
  float4* acc = ffs_smem + FFS_V * 2 * N;  // [FFS_V][N]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float hl2 = -0.34657359027997264f;  // -ln(2)/2: -log|r| = hl2 log2|r|^2
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.ntile) break;
    const int2 tij = a.tiles[t];
    const int I = tij.x, J = tij.y;
    const int i0 = I * FFS_V, nI = min(FFS_V, a.M - i0);
    const int j0 = J * FFS_V, nJ = min(FFS_V, a.M - j0);
    const bool diag = I == J;
    const int64_t p0 = (int64_t)j0 * N;
    for (int e = threadIdx.x; e < nJ * 2 * N; e += blockDim.x) {
      const int b = e / (2 * N), rem = e - b * 2 * N;
      col[e] = src[p0 + b * N + 32 * (rem >> 6) + (rem & 31)];
    }
    for (int e = threadIdx.x; e < nJ * N; e += blockDim.x) acc[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const bool rot = nJ >= FFS_W;
    const int K = rot ? nJ : nJ + FFS_W - 1;
    for (int r0 = 0; r0 < nI; r0 += FFS_W) {
      const int ai = r0 + w;
      const bool arow = ai < nI;
      const int av = i0 + ai;
      float4 rp[R];
      float gxs[R], gys[R], sxr[R], cxr[R], syr[R], cyr[R];
      float4 ca = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 ha = make_float2(0.f, 0.f);
      if (arow) {
        ca = centre32[av];
        ha = h2[av];
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        rp[r] = arow ? src[(int64_t)av * N + lane + 32 * r] : make_float4(0.f, 0.f, 0.f, 0.f);
        gxs[r] = hl2 * rp[r].z;
        gys[r] = hl2 * rp[r].w;
        sxr[r] = cxr[r] = syr[r] = cyr[r] = 0.f;
      }
      const float reach_a = sqrtf(ha.y);
      for (int k = 0; k < K; ++k) {
        int bj = rot ? w + k : k - w;
        if (rot && bj >= nJ) bj -= nJ;
        if (arow && bj >= 0 && bj < nJ && (!diag || bj > ai)) {
          const int bv = j0 + bj;
          const float4 cb = centre32[bv];
          const float2 hb = h2[bv];
          const float dx = (ca.x - cb.x) + (ca.z - cb.z), dy = (ca.y - cb.y) + (ca.w - cb.w);
          float tx[R], ty[R], lx[R], ly[R], ax[R], ay[R], mr[R], ux[R], uy[R], mc[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            tx[r] = dx + rp[r].x;
            ty[r] = dy + rp[r].y;
            lx[r] = ly[r] = ax[r] = ay[r] = ux[r] = uy[r] = 0.f;
            mr[r] = mc[r] = 3.0e38f;
          }
          // the minima are needed only when the reach circles of A and B overlap
          const float rs = reach_a + sqrtf(hb.y);
          const bool test = a.near_mask && fmaf(dx, dx, dy * dy) <= rs * rs;
          const float4* colB = col + bj * 2 * N;
          if (test)
            ffs_pair<R, true>(colB, lane, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
          else
            ffs_pair<R, false>(colB, lane, tx, ty, rp, gxs, gys, lx, ly, ax, ay, mr, ux, uy, mc);
#pragma unroll
          for (int r = 0; r < R; ++r) {  // targets of A, source vesicle B
            if (test && mr[r] <= hb.x) {
              ffs_near(a, (int64_t)av * N + lane + 32 * r, bv);
            } else {
              neumaier_add(sxr[r], cxr[r], fmaf(hl2, lx[r], ax[r]));
              neumaier_add(syr[r], cyr[r], fmaf(hl2, ly[r], ay[r]));
            }
          }
#pragma unroll
          for (int c = 0; c < R; ++c) {  // targets of B, source vesicle A
            if (test && mc[c] <= ha.x) {
              ffs_near(a, (int64_t)bv * N + lane + 32 * c, av);
            } else {
              float4& v = acc[bj * N + lane + 32 * c];
              float4 s = v;
              neumaier_add(s.x, s.y, ux[c]);
              neumaier_add(s.z, s.w, uy[c]);
              v = s;
            }
          }
        }
        __syncthreads();
      }
      if (arow) {
        if (diag) {  // chunk I = J: the row sums join the column accumulators of A's points
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float4& v = acc[ai * N + lane + 32 * r];
            float4 s = v;
            neumaier_add(s.x, s.y, sxr[r]);
            s.y += cxr[r];
            neumaier_add(s.z, s.w, syr[r]);
            s.w += cyr[r];
            v = s;
          }
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r)
            a.part[(int64_t)J * a.P + (int64_t)av * N + lane + 32 * r] = make_float4(sxr[r], cxr[r], syr[r], cyr[r]);
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < nJ * N; e += blockDim.x) {  // chunk I's contributions to chunk J's points
      const float4 v = acc[e];
      a.part[(int64_t)I * a.P + p0 + e] = v;
    }
    __syncthreads();
  }
}

// u (CSR blocks [u_x(N), u_y(N)] per vesicle) += sum over chunks of part, in chunk order (double-float); near
// counts clamped to MAX_NEAR and each near list sorted ascending.
__global__ void __launch_bounds__(256) k_farfield_sym_reduce(FfSymArgs a, double* __restrict__ u) {
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
  const int64_t v = p / a.N;
  const int64_t to = v * a.N;
  const int64_t loc = p - to;
  u[2 * to + loc] += sx;
  u[2 * to + a.N + loc] += sy;
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

}  // namespace vs
