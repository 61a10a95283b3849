// Cluster tree for the multipole far field (VS_FLAG_FARFIELD_TREE, plan precision 4). The paper names the
// fast multipole method as the route to a far field whose cost grows linearly with the number of vesicles
// (Sec. 4.1, Sec. 4.5); the vesicle multipole mode (k_farfield_loc.cuh) still tests and translates every
// pair of vesicles. Here the vesicles are grouped in a quadtree of their centres and a target vesicle takes
// whole clusters through one multipole-to-local translation each, so the translations per target grow like
// log M instead of M.
//
// Tree (k_tree_build, one CTA): Morton keys of the vesicle centres on a 2^16 x 2^16 grid over their bounding
// square, sorted in shared memory (bitonic); level l + 1 splits every box of level l holding more than
// TREE_LEAF vesicles by the next two bits of the key. A box is a range of the sorted vesicles; the boxes of a
// level are consecutive, children in key order.
//
// Cluster expansions (k_tree_moments: all leaves at once, then the internal boxes level by level upwards): a box's centre is the mean of its vesicles'
// centres and its radius bounds every point of them. Its moments A_k, B_k, D_k about its centre follow
// exactly from those of its members (vesicles for a leaf, child boxes otherwise) about theirs: with
// s = s' + delta, delta the member's centre minus the box centre,
//   A_k = sum_j C(k, j) delta^(k-j) A'_j,   B_k = sum_j C(k, j) conj(delta)^(k-j) B'_j,
//   D_k = sum_j C(k, j) conj(delta)^(k-j) (D'_j + delta conj(A'_j))
// (the multipole-to-multipole shift; finite sums, FP64). Their expansion coefficients follow as for a vesicle.
//
// Walk (k_ff_local_tree, one CTA per target vesicle A): from the root, a box that passes the vesicle test
// |c_A - c_B| > 2 (reach_A + radius_B) is translated whole into A's local expansion; a leaf that does not
// pass hands its vesicles to the vesicle test, which translates them or lists them for point sums; other
// boxes open their children. Every vesicle of a box that passes also passes the vesicle test (its centre is
// within radius_B - reach_v of c_B), so the listed vesicles are exactly those of k_ff_local and the
// truncation error per source is bounded as there. Lists are compacted by block scans in walk order, so the
// sums are deterministic. A target whose frontier or lists outgrow shared memory takes k_ff_local's loop
// over all vesicles instead.
#pragma once
#include "k_farfield_loc.cuh"

namespace vs {

constexpr int TREE_MAX_M = 16384;  // vesicles (one CTA sorts their keys in shared memory)
constexpr int TREE_LEAF = 8;       // a box of more vesicles is split, down to TREE_LMAX levels
constexpr int TREE_LMAX = 16;      // 16 bits of cell coordinate per axis
constexpr int TREE_THREADS = 1024;
constexpr int TREE_FR = 256;  // boxes per frontier of a walk
constexpr int TREE_BL = 512;  // separated boxes per target vesicle
constexpr int TREE_CL = 256;  // vesicles of the unseparated leaves per target vesicle
constexpr int TREE_K = FF_MP_P + 2;  // moments of each kind
// Boxes: an internal box holds more than TREE_LEAF vesicles, so a level has at most M / (TREE_LEAF + 1)
// of them and each has at most 4 children.
inline int64_t tree_max_boxes(int M) { return 1 + 4 * (int64_t)(TREE_LMAX + 1) * (M / (TREE_LEAF + 1) + 1); }
inline size_t tree_build_smem(int M) {
  size_t k = 1;
  while ((int)k < M) k <<= 1;
  return k * sizeof(unsigned long long);
}

struct FfTreeArgs {
  int M;
  int64_t max_boxes;
  const double2* vcen;  // [M] vesicle centres (FP64)
  const float4* vcen32; // [M] as float hi/lo
  const float2* vh2;    // [M] (h^2, reach^2)
  const double2* vraw;  // [M][3 TREE_K] moments A, B, D about the vesicle centre
  int* order;           // [M] vesicles in key order
  int* owner;           // [M] box of each sorted position while the tree is built
  int* lstart;          // [TREE_LMAX + 2] first box of each level; the last entry: number of boxes
  int2* range;          // [boxes] sorted positions [lo, hi)
  int* parent;          // [boxes]
  int* first;           // [boxes] first child
  int* nchild;          // [boxes] 0 for a leaf
  double2* bcen;        // [boxes] centre
  float4* bcen32;       // [boxes] centre as float hi/lo
  float* brad;          // [boxes] radius
  double2* braw;        // [boxes][3 TREE_K] moments about the box centre
  float4* bcoef;        // [boxes][2 (FF_MP_P + 1)] expansion coefficients
  float2* ba0;          // [boxes]
};

__device__ __forceinline__ unsigned tree_spread(unsigned x) {  // 16 bits to the even bit positions
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Exclusive prefix sum over the CTA of one value per thread (warp shuffles, then the warps' totals from sw,
// 32 entries); returns the thread's offset and the CTA's total in *tot. Every thread of the CTA calls it.
template <typename T>
__device__ __forceinline__ T tree_scan(T v, T* sw, T* tot) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sw[wid] = x;
  __syncthreads();
  T base = 0, all = 0;
  for (int w = 0; w < nw; ++w) {
    const T s = sw[w];
    if (w < wid) base += s;
    all += s;
  }
  *tot = all;
  __syncthreads();  // sw is free for the next scan
  return base + x - v;
}

// Position i of the sorted keys opens a child box at level l + 1 (its box b at level l is split).
__device__ __forceinline__ bool tree_opens(const unsigned long long* key, int i, int lo, int shift) {
  if (i == lo) return true;
  return ((unsigned)(key[i] >> 32) >> shift & 3u) != ((unsigned)(key[i - 1] >> 32) >> shift & 3u);
}

__global__ void __launch_bounds__(TREE_THREADS) k_tree_build(FfTreeArgs t) {
  extern __shared__ unsigned long long key[];
  __shared__ double red[4][TREE_THREADS / 32];
  __shared__ int sw[32];
  const int M = t.M, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int K2 = 1;
  while (K2 < M) K2 <<= 1;
  // bounding square of the centres
  double x0 = 1e300, y0 = 1e300, x1 = -1e300, y1 = -1e300;
  for (int v = tid; v < M; v += TREE_THREADS) {
    const double2 c = t.vcen[v];
    x0 = fmin(x0, c.x); y0 = fmin(y0, c.y); x1 = fmax(x1, c.x); y1 = fmax(y1, c.y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, o)); y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, o));
    x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, o)); y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, o));
  }
  if (lane == 0) { red[0][wid] = x0; red[1][wid] = y0; red[2][wid] = x1; red[3][wid] = y1; }
  __syncthreads();
  x0 = red[0][0]; y0 = red[1][0]; x1 = red[2][0]; y1 = red[3][0];
  for (int w = 1; w < TREE_THREADS / 32; ++w) {
    x0 = fmin(x0, red[0][w]); y0 = fmin(y0, red[1][w]); x1 = fmax(x1, red[2][w]); y1 = fmax(y1, red[3][w]);
  }
  const double side = fmax(x1 - x0, y1 - y0);
  const double sc16 = side > 0.0 ? 65535.0 / side : 0.0;
  for (int i = tid; i < K2; i += TREE_THREADS) {
    unsigned long long k = ~0ull;
    if (i < M) {
      const double2 c = t.vcen[i];
      const unsigned qx = (unsigned)fmin(65535.0, fmax(0.0, floor((c.x - x0) * sc16)));
      const unsigned qy = (unsigned)fmin(65535.0, fmax(0.0, floor((c.y - y0) * sc16)));
      k = ((unsigned long long)(tree_spread(qx) | (tree_spread(qy) << 1)) << 32) | (unsigned)i;
    }
    key[i] = k;
  }
  __syncthreads();
  // bitonic sort, ascending (keys are distinct: the low word is the vesicle index)
  for (int size = 2; size <= K2; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int p = tid; p < K2 / 2; p += TREE_THREADS) {
        const int lo = 2 * p - (p & (stride - 1)), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = key[lo], b = key[hi];
        if ((a > b) == up) { key[lo] = b; key[hi] = a; }
      }
      __syncthreads();
    }
  for (int i = tid; i < M; i += TREE_THREADS) {
    t.order[i] = (int)(key[i] & 0xffffffffull);
    t.owner[i] = 0;
  }
  if (tid == 0) {
    t.range[0] = make_int2(0, M);
    t.parent[0] = -1;
    t.first[0] = 0;
    t.nchild[0] = 0;
    t.lstart[0] = 0;
    t.lstart[1] = 1;
  }
  __syncthreads();
  // levels: each thread takes a contiguous run of sorted positions
  const int per = (M + TREE_THREADS - 1) / TREE_THREADS;
  const int i0 = min(M, tid * per), i1 = min(M, i0 + per);
  int ls = 0, le = 1, level = 0;
  for (; level < TREE_LMAX; ++level) {
    const int shift = 2 * (15 - level);
    int cnt = 0;
    for (int i = i0; i < i1; ++i) {
      const int b = t.owner[i];
      if (b < ls) continue;  // a leaf of an earlier level
      const int2 r = t.range[b];
      if (r.y - r.x > TREE_LEAF && tree_opens(key, i, r.x, shift)) ++cnt;
    }
    int total;
    int run = tree_scan(cnt, sw, &total);
    if (total == 0 || le + total > t.max_boxes) break;  // (the bound on the boxes is never reached)
    for (int i = i0; i < i1; ++i) {
      const int b = t.owner[i];
      if (b < ls) continue;
      const int2 r = t.range[b];
      if (r.y - r.x <= TREE_LEAF) continue;
      if (tree_opens(key, i, r.x, shift)) {
        const int c = le + run++;
        t.range[c].x = i;
        t.parent[c] = b;
        if (i == r.x) t.first[b] = c;
        atomicAdd(&t.nchild[b], 1);
      }
      t.owner[i] = le + run - 1;
    }
    __syncthreads();
    for (int c = le + tid; c < le + total; c += TREE_THREADS) {
      const int b = t.parent[c];
      t.range[c].y = (c + 1 < le + total && t.parent[c + 1] == b) ? t.range[c + 1].x : t.range[b].y;
      t.first[c] = 0;
      t.nchild[c] = 0;
    }
    ls = le;
    le += total;
    if (tid == 0) t.lstart[level + 2] = le;
    __syncthreads();
  }
  for (int l = level + 2 + tid; l <= TREE_LMAX + 1; l += TREE_THREADS) t.lstart[l] = le;
}

// Binomial coefficients C(k, j), k, j < TREE_K, fixed at compile time (exact in FP64): the shifts below read
// them instead of dividing in FP64, whose long latency at 1/64 of the FP32 rate sat on each box's critical path.
struct TreeBinom {
  double c[TREE_K][TREE_K];
};
__host__ __device__ constexpr TreeBinom tree_binom_table() {
  TreeBinom t{};
  for (int k = 0; k < TREE_K; ++k)
    for (int j = 0; j < TREE_K; ++j) {
      double c = j <= k ? 1.0 : 0.0;
      for (int i = 1; i <= j && j <= k; ++i) c = c * (k - j + i) / i;
      t.c[k][j] = c;
    }
  return t;
}
__constant__ TreeBinom c_tree_binom = tree_binom_table();

// Moments, centre and radius of boxes from their members: with leaves set, every leaf box of the tree at
// once (its members are vesicles, whose moments are known); otherwise the internal boxes of one level, deepest
// level first. One CTA per box (grid-stride), a thread per (member, moment) so that the FP64 shifts of up to
// TREE_LEAF members run side by side; the members' sums are added in member order. Members beyond TREE_LEAF
// (coincident vesicles in a leaf at the deepest level) are taken in further rounds by the same threads.
constexpr int TM_THREADS = 3 * TREE_K * TREE_LEAF;

__global__ void __launch_bounds__(TM_THREADS) k_tree_moments(FfTreeArgs t, int level, int leaves) {
  constexpr int K = TREE_K, MC = TREE_LEAF, NO = 3 * K;
  __shared__ double2 sm[NO];
  __shared__ double2 part[MC][NO];
  __shared__ double2 mc[MC];
  __shared__ double mr[MC], mw[MC];
  __shared__ double bn[K][K];
  __shared__ double2 cen;
  const int b0 = leaves ? 0 : t.lstart[level], b1 = leaves ? t.lstart[TREE_LMAX + 1] : t.lstart[level + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < K * K; e += blockDim.x) bn[e / K][e % K] = c_tree_binom.c[e / K][e % K];

  for (int b = b0 + blockIdx.x; b < b1; b += gridDim.x) {
    const int nc = t.nchild[b];
    if ((nc == 0) != (leaves != 0)) continue;  // uniform over the CTA
    const int2 r = t.range[b];
    const bool leaf = nc == 0;
    const int nm = leaf ? r.y - r.x : nc;
    if (tid < nm && tid < MC) {
      const int id = leaf ? t.order[r.x + tid] : t.first[b] + tid;
      mc[tid] = leaf ? t.vcen[id] : t.bcen[id];
      mr[tid] = leaf ? sqrt((double)t.vh2[id].y) : (double)t.brad[id];
      mw[tid] = leaf ? 1.0 : (double)(t.range[id].y - t.range[id].x);
    }
    __syncthreads();
    if (tid == 0) {  // centre: mean of the vesicle centres (children weighted by their counts), in order
      double cx = 0.0, cy = 0.0;
      for (int m = 0; m < nm; ++m) {
        const int id = m < MC ? 0 : (leaf ? t.order[r.x + m] : t.first[b] + m);
        const double2 c = m < MC ? mc[m] : (leaf ? t.vcen[id] : t.bcen[id]);
        const double w = m < MC ? mw[m] : (leaf ? 1.0 : (double)(t.range[id].y - t.range[id].x));
        cx += w * c.x;
        cy += w * c.y;
      }
      const double inv = 1.0 / (double)(r.y - r.x);
      cx *= inv;
      cy *= inv;
      double rr = 0.0;
      for (int m = 0; m < nm; ++m) {
        const int id = m < MC ? 0 : (leaf ? t.order[r.x + m] : t.first[b] + m);
        const double2 c = m < MC ? mc[m] : (leaf ? t.vcen[id] : t.bcen[id]);
        const double rm = m < MC ? mr[m] : (leaf ? sqrt((double)t.vh2[id].y) : (double)t.brad[id]);
        rr = fmax(rr, sqrt((c.x - cx) * (c.x - cx) + (c.y - cy) * (c.y - cy)) + rm);
      }
      cen = make_double2(cx, cy);
      t.bcen[b] = cen;
      const float hx = (float)cx, hy = (float)cy;
      t.bcen32[b] = make_float4(hx, hy, (float)(cx - (double)hx), (float)(cy - (double)hy));
      t.brad[b] = (float)rr * (1.f + 1e-6f);
    }
    __syncthreads();
    const int ml = tid / NO, o = tid - ml * NO;
    const int kind = o / K, k = o - kind * K;
    double sr = 0.0, si = 0.0;
    for (int m = ml; m < nm; m += MC) {
      const int id = leaf ? t.order[r.x + m] : t.first[b] + m;
      const double2 c = leaf ? t.vcen[id] : t.bcen[id];
      const double2* mo = (leaf ? t.vraw : t.braw) + (int64_t)id * 3 * K;
      const double dr = c.x - cen.x, di = c.y - cen.y;  // delta
      const double wr = dr, wi = kind == 0 ? di : -di;   // delta or conj(delta)
      // sum_j C(k, j) w^(k - j) X_j, with X_j = A_j, B_j, or D_j + delta conj(A_j)
      double pr = 1.0, pi = 0.0;  // w^(k - j), from j = k down to 0
      for (int j = k; j >= 0; --j) {
        double xr, xi;
        if (kind == 0) {
          xr = mo[j].x;
          xi = mo[j].y;
        } else if (kind == 1) {
          xr = mo[K + j].x;
          xi = mo[K + j].y;
        } else {
          const double2 a = mo[j], d = mo[2 * K + j];
          xr = d.x + (dr * a.x + di * a.y);  // delta conj(A_j)
          xi = d.y + (di * a.x - dr * a.y);
        }
        const double c = bn[k][j];
        sr = fma(c, pr * xr - pi * xi, sr);
        si = fma(c, pr * xi + pi * xr, si);
        const double nr = pr * wr - pi * wi;
        pi = pr * wi + pi * wr;
        pr = nr;
      }
    }
    part[ml][o] = make_double2(sr, si);
    __syncthreads();
    if (tid < NO) {
      double2 x = part[0][tid];
      for (int m = 1; m < MC && m < nm; ++m) {
        x.x += part[m][tid].x;
        x.y += part[m][tid].y;
      }
      sm[tid] = x;
      t.braw[(int64_t)b * 3 * K + tid] = x;
    }
    __syncthreads();
    ffm_coef<FF_MP_P>(tid, sm, sm + K, sm + 2 * K, t.bcoef + (int64_t)b * 2 * (FF_MP_P + 1), t.ba0 + b);
    __syncthreads();
  }
}

// One CTA of 128 threads per target vesicle: the walk above, then the translations of the separated boxes
// and vesicles in list order (thread j takes items j, j + 128, ...) and the list of the others, ascending.
template <int P>
__global__ void __launch_bounds__(128) k_ff_local_tree(FfLocArgs a, FfTreeArgs t) {
  constexpr int NT = P + 1, NF = ffl_floats(P);
  __shared__ int fr[2][TREE_FR];
  __shared__ int bl[TREE_BL];
  __shared__ int cl[TREE_CL];
  __shared__ unsigned long long sw64[4];
  __shared__ int sw[4];
  __shared__ int s_nfr, s_nbl, s_ncl, s_nnext, s_over;
  const int A = blockIdx.x, tid = threadIdx.x;
  const float4 ca = a.centre32[A];
  const float ra = sqrtf(a.h2[A].y);
  if (tid == 0) {
    fr[0][0] = 0;
    s_nfr = 1; s_nbl = 0; s_ncl = 0; s_nnext = 0; s_over = 0;
  }
  __syncthreads();
  int cur = 0;
  while (s_nfr > 0 && !s_over) {
    const int n = s_nfr;
    for (int base = 0; base < n; base += 128) {
      const int idx = base + tid;
      int kind = 0, cnt = 0, b = 0;  // kind 1: separated box; 2: leaf (cnt vesicles); 3: cnt children
      if (idx < n) {
        b = fr[cur][idx];
        float dx, dy;
        if (ffl_separated(ca, ra, t.bcen32[b], t.brad[b], dx, dy)) {
          kind = 1;
        } else if (t.nchild[b] == 0) {
          kind = 2;
          cnt = t.range[b].y - t.range[b].x;
        } else {
          kind = 3;
          cnt = t.nchild[b];
        }
      }
      // one scan of the three counts packed as (separated boxes | children << 16 | leaf vesicles << 32)
      typedef unsigned long long u64;
      u64 tot;
      const u64 mine = (u64)(kind == 1 ? 1 : 0) | ((u64)(kind == 3 ? cnt : 0) << 16) |
                       ((u64)(kind == 2 ? cnt : 0) << 32);
      const u64 ex = tree_scan<u64>(mine, sw64, &tot);
      const int o1 = (int)(ex & 0xffffu), o3 = (int)((ex >> 16) & 0xffffu), o2 = (int)(ex >> 32);
      const int tot1 = (int)(tot & 0xffffu), tot3 = (int)((tot >> 16) & 0xffffu), tot2 = (int)(tot >> 32);
      const int nbl = s_nbl, ncl = s_ncl, nnx = s_nnext;
      if (kind == 1 && nbl + o1 < TREE_BL) bl[nbl + o1] = b;
      if (kind == 2)
        for (int q = 0; q < cnt && ncl + o2 + q < TREE_CL; ++q) cl[ncl + o2 + q] = t.order[t.range[b].x + q];
      if (kind == 3)
        for (int q = 0; q < cnt && nnx + o3 + q < TREE_FR; ++q) fr[cur ^ 1][nnx + o3 + q] = t.first[b] + q;
      __syncthreads();
      if (tid == 0) {
        s_nbl = nbl + tot1;
        s_ncl = ncl + tot2;
        s_nnext = nnx + tot3;
        if (s_nbl > TREE_BL || s_ncl > TREE_CL || s_nnext > TREE_FR) s_over = 1;
      }
      __syncthreads();
      if (s_over) break;
    }
    if (tid == 0) {
      s_nfr = s_nnext;
      s_nnext = 0;
    }
    cur ^= 1;
    __syncthreads();
  }
  if (s_over) {  // uniform: every vesicle tested and translated one by one
    ffl_local_all<P>(a, A);
    return;
  }
  // the vesicles of the unseparated leaves: separated ones join the translations (after the boxes, in bl's
  // tail), the others are listed
  const int nbox = s_nbl, ncand = s_ncl;
  __shared__ int nl[TREE_CL];
  __shared__ int s_nv, s_nl;
  if (tid == 0) { s_nv = 0; s_nl = 0; }
  __syncthreads();
  for (int base = 0; base < ncand; base += 128) {
    const int idx = base + tid;
    int sep = 0, lst = 0, B = -1;
    if (idx < ncand) {
      B = cl[idx];
      float dx, dy;
      if (B != A) {
        if (ffl_separated(ca, ra, a.centre32[B], sqrtf(a.h2[B].y), dx, dy)) sep = 1;
        else lst = 1;
      }
    }
    int tboth;
    const int both = tree_scan<int>(sep | (lst << 16), sw, &tboth);  // separated | listed << 16
    const int ov = both & 0xffff, ol = both >> 16, tv = tboth & 0xffff, tl = tboth >> 16;
    const int nv = s_nv, nlc = s_nl;
    if (sep) cl[nv + ov] = B;  // compacted in place: position nv + ov <= idx, every read of cl above done
    if (lst) nl[nlc + ol] = B;
    __syncthreads();
    if (tid == 0) { s_nv = nv + tv; s_nl = nlc + tl; }
    __syncthreads();
  }
  const int nves = s_nv, nlist = s_nl;
  float acc[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) acc[i] = 0.f;
  for (int j = tid; j < nbox + nves; j += 128) {
    float dx, dy;
    if (j < nbox) {
      const int b = bl[j];
      ffl_separated(ca, ra, t.bcen32[b], t.brad[b], dx, dy);
      ffl_translate<P>(acc, dx, dy, t.bcoef + (int64_t)b * 2 * NT, t.ba0[b]);
    } else {
      const int B = cl[j - nbox];
      ffl_separated(ca, ra, a.centre32[B], sqrtf(a.h2[B].y), dx, dy);
      ffl_translate<P>(acc, dx, dy, a.coef + (int64_t)B * 2 * NT, a.a0[B]);
    }
  }
  ffl_store<P>(acc, a.loc + (int64_t)A * NF);
  // listed vesicles in ascending order (rank of each among the distinct indices)
  for (int i = tid; i < nlist; i += 128) {
    const int B = nl[i];
    int rank = 0;
    for (int q = 0; q < nlist; ++q) rank += nl[q] < B;
    if (rank < FFL_LIST) a.nlist[(int64_t)A * FFL_LIST + rank] = B;
  }
  if (tid == 0) a.ncnt[A] = nlist;
}

}  // namespace vs
