// Batched FP64 dense kernels for the per-vesicle operators (Eqs. bending_op .. PTop, Sec. 3.1).
//
// Every vesicle owns a row-major matrix scratch (MatLayout). The products that define the
// operators are computed by one batched GEMM whose operands are read through small functor
// structs, so diagonal scalings and the differentiation circulant are applied on the fly:
//   T  = S Ten,          Ten = [D_s diag(x_s); D_s diag(y_s)]             (2N x N)
//   L  = P T,            P   = [diag(x_s) D_s, diag(y_s) D_s]             (N x N)
//   D4 = (D_s D_s)(D_s D_s)                                               (N x N)
//   B  = -kappa S blockdiag(D4, D4)                                       (2N x 2N)
//   W  = P B, then W <- L^{-1} W                                          (N x 2N)
// (FP32 path: W = L^{-1} (P B) with the explicit FP32 inverse of L, see k_gj_inverse)
//   A  = I - dt (B - T W) = I - dt (I - T L^{-1} P) B                     (2N x 2N)
// with D_s = diag(1/|X_alpha|) D_alpha.
#pragma once
#include "common.cuh"

namespace vs {

struct OpCtx {
  VesIndex vi;
  const double* tab;
  const double* sa;
  const double* tx;
  const double* ty;
  double* scratch;
  float* scratch32;  // FP32 copies with the same per-vesicle layout (mixed-precision path)
  const float* tab32;   // FP32 copy of tab
  const float4* g32;    // FP32 (1/|X_alpha|, x_s, y_s, 0) per point
  __device__ __forceinline__ double* mat(int v, int N, int64_t sub) const {
    return scratch + vi.moff[v] + sub * (int64_t)N * N;
  }
  __device__ __forceinline__ float* mat32(int v, int N, int64_t sub) const {
    return scratch32 + vi.moff[v] + sub * (int64_t)N * N;
  }
  __device__ __forceinline__ double dcirc(int v, int N, int m) const {
    m %= N;
    if (m < 0) m += N;
    return tab[vi.toff[v] + m];
  }
  // FP32 circulant entry d(m) for m in (-N, N)
  __device__ __forceinline__ float dcirc32(int v, int N, int m) const { return tab32[vi.toff[v] + (m < 0 ? m + N : m)]; }
};

// FP32 entry (i, k) of P = [diag(x_s) D_s, diag(y_s) D_s] (N x 2N), all arithmetic in FP32
__device__ __forceinline__ float p_entry32(const OpCtx& c, int v, int N, int i, int k) {
  const float4 g = c.g32[c.vi.off[v] + i];
  const int kk = (k < N) ? k : k - N;
  return ((k < N) ? g.y : g.z) * g.x * c.dcirc32(v, N, i - kk);
}

// T = S Ten at slot s.
struct OpT {
  using T = double;
  OpCtx c; int s;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = N; k = 2 * N; }
  __device__ double a(int v, int N, int i, int k) const {
    const int64_t o = c.vi.off[v];
    return c.mat(v, N, MatLayout::slot(s) + MatLayout::S)[(int64_t)i * 2 * N + k] / c.sa[o + (k % N)];
  }
  __device__ double b(int v, int N, int k, int j) const {
    const int64_t o = c.vi.off[v];
    const double t = (k < N) ? c.tx[o + j] : c.ty[o + j];
    return c.dcirc(v, N, (k % N) - j) * t;
  }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)i * N + j] = acc;
  }
};

// P row i, column k (k < 2N): (x_s or y_s)_i d((i - k mod N)) / sa_i
__device__ __forceinline__ double p_entry(const OpCtx& c, int v, int N, int i, int k) {
  const int64_t o = c.vi.off[v];
  const double t = (k < N) ? c.tx[o + i] : c.ty[o + i];
  return t * c.dcirc(v, N, i - (k % N)) / c.sa[o + i];
}

// L = P T at slot s.
struct OpL {
  using T = double;
  OpCtx c; int s;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = 2 * N; }
  __device__ double a(int v, int N, int i, int k) const { return p_entry(c, v, N, i, k); }
  __device__ double b(int v, int N, int k, int j) const {
    return c.mat(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)k * N + j];
  }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::slot(s) + MatLayout::L)[(int64_t)i * N + j] = acc;
  }
};

// D2 = D_s D_s, written to the A region (scratch).
struct OpD2 {
  using T = double;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = N; }
  __device__ double a(int v, int N, int i, int k) const {
    return c.dcirc(v, N, i - k) / c.sa[c.vi.off[v] + i];
  }
  __device__ double b(int v, int N, int k, int j) const {
    return c.dcirc(v, N, k - j) / c.sa[c.vi.off[v] + k];
  }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::A)[(int64_t)i * N + j] = acc;
  }
};

// D4 = D2 D2.
struct OpD4 {
  using T = double;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = N; }
  __device__ double a(int v, int N, int i, int k) const { return c.mat(v, N, MatLayout::A)[(int64_t)i * N + k]; }
  __device__ double b(int v, int N, int k, int j) const { return c.mat(v, N, MatLayout::A)[(int64_t)k * N + j]; }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::D4)[(int64_t)i * N + j] = acc;
  }
};

// B[:, h N + j] = -kappa sum_k S[i][h N + k] D4[k][j] with S from slot s.
struct OpB {
  using T = double;
  OpCtx c; int s; int h; double kappa;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = N; k = N; }
  __device__ double a(int v, int N, int i, int k) const {
    return c.mat(v, N, MatLayout::slot(s) + MatLayout::S)[(int64_t)i * 2 * N + h * N + k];
  }
  __device__ double b(int v, int N, int k, int j) const { return c.mat(v, N, MatLayout::D4)[(int64_t)k * N + j]; }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::B)[(int64_t)i * 2 * N + h * N + j] = -kappa * acc;
  }
};

// W = P B (N x 2N).
struct OpPB {
  using T = double;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = 2 * N; k = 2 * N; }
  __device__ double a(int v, int N, int i, int k) const { return p_entry(c, v, N, i, k); }
  __device__ double b(int v, int N, int k, int j) const { return c.mat(v, N, MatLayout::B)[(int64_t)k * 2 * N + j]; }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    c.mat(v, N, MatLayout::W)[(int64_t)i * 2 * N + j] = acc;
  }
};

// A = I - dt (B - T W) with T from slot s.
struct OpA {
  using T = double;
  OpCtx c; int s; double dt;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = 2 * N; k = N; }
  __device__ double a(int v, int N, int i, int k) const {
    return c.mat(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)i * N + k];
  }
  __device__ double b(int v, int N, int k, int j) const { return c.mat(v, N, MatLayout::W)[(int64_t)k * 2 * N + j]; }
  __device__ void store(int v, int N, int i, int j, double acc) const {
    const double bij = c.mat(v, N, MatLayout::B)[(int64_t)i * 2 * N + j];
    c.mat(v, N, MatLayout::A)[(int64_t)i * 2 * N + j] = ((i == j) ? 1.0 : 0.0) - dt * (bij - acc);
  }
};

// ---- FP32 operator products (mixed-precision path): the same products from the FP32 copy of S,
// used only to build factorisations that precondition FP64 matrix-free refinement.
struct OpT32 {
  using T = float;
  OpCtx c; int s;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = N; k = 2 * N; }
  __device__ float a(int v, int N, int i, int k) const {
    return c.mat32(v, N, MatLayout::slot(s) + MatLayout::S)[(int64_t)i * 2 * N + k] *
           c.g32[c.vi.off[v] + ((k < N) ? k : k - N)].x;
  }
  __device__ float b(int v, int N, int k, int j) const {
    const float4 g = c.g32[c.vi.off[v] + j];
    return c.dcirc32(v, N, ((k < N) ? k : k - N) - j) * ((k < N) ? g.y : g.z);
  }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)i * N + j] = acc;
  }
};
struct OpL32 {
  using T = float;
  OpCtx c; int s;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = 2 * N; }
  __device__ float a(int v, int N, int i, int k) const { return p_entry32(c, v, N, i, k); }
  __device__ float b(int v, int N, int k, int j) const {
    return c.mat32(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)k * N + j];
  }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::slot(s) + MatLayout::L)[(int64_t)i * N + j] = acc;
  }
};
struct OpD2_32 {
  using T = float;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = N; }
  __device__ float a(int v, int N, int i, int k) const { return c.dcirc32(v, N, i - k) * c.g32[c.vi.off[v] + i].x; }
  __device__ float b(int v, int N, int k, int j) const { return c.dcirc32(v, N, k - j) * c.g32[c.vi.off[v] + k].x; }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::A)[(int64_t)i * N + j] = acc;
  }
};
struct OpD4_32 {
  using T = float;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = N; }
  __device__ float a(int v, int N, int i, int k) const { return c.mat32(v, N, MatLayout::A)[(int64_t)i * N + k]; }
  __device__ float b(int v, int N, int k, int j) const { return c.mat32(v, N, MatLayout::A)[(int64_t)k * N + j]; }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::D4)[(int64_t)i * N + j] = acc;
  }
};
struct OpB32 {
  using T = float;
  OpCtx c; int s; int h; double kappa;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = N; k = N; }
  __device__ float a(int v, int N, int i, int k) const {
    return c.mat32(v, N, MatLayout::slot(s) + MatLayout::S)[(int64_t)i * 2 * N + h * N + k];
  }
  __device__ float b(int v, int N, int k, int j) const { return c.mat32(v, N, MatLayout::D4)[(int64_t)k * N + j]; }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::B)[(int64_t)i * 2 * N + h * N + j] = (float)(-kappa) * acc;
  }
};
struct OpPB32 {
  using T = float;
  OpCtx c;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = 2 * N; k = 2 * N; }
  __device__ float a(int v, int N, int i, int k) const { return p_entry32(c, v, N, i, k); }
  __device__ float b(int v, int N, int k, int j) const { return c.mat32(v, N, MatLayout::B)[(int64_t)k * 2 * N + j]; }
  __device__ void store(int v, int N, int i, int j, float acc) const {  // P B parked in the A block
    c.mat32(v, N, MatLayout::A)[(int64_t)i * 2 * N + j] = acc;
  }
};
// W = L^{-1} (P B) with the FP32 inverse of L (held in the L block of slot s).
struct OpW32 {
  using T = float;
  OpCtx c; int s;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = 2 * N; k = N; }
  __device__ float a(int v, int N, int i, int k) const {
    return c.mat32(v, N, MatLayout::slot(s) + MatLayout::L)[(int64_t)i * N + k];
  }
  __device__ float b(int v, int N, int k, int j) const { return c.mat32(v, N, MatLayout::A)[(int64_t)k * 2 * N + j]; }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    c.mat32(v, N, MatLayout::W)[(int64_t)i * 2 * N + j] = acc;
  }
};
struct OpA32 {
  using T = float;
  OpCtx c; int s; double dt;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = 2 * N; n = 2 * N; k = N; }
  __device__ float a(int v, int N, int i, int k) const {
    return c.mat32(v, N, MatLayout::slot(s) + MatLayout::T)[(int64_t)i * N + k];
  }
  __device__ float b(int v, int N, int k, int j) const { return c.mat32(v, N, MatLayout::W)[(int64_t)k * 2 * N + j]; }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    const float bij = c.mat32(v, N, MatLayout::B)[(int64_t)i * 2 * N + j];
    c.mat32(v, N, MatLayout::A)[(int64_t)i * 2 * N + j] = ((i == j) ? 1.f : 0.f) - (float)dt * (bij - acc);
  }
};

// N x N blocks inside the FP32 scratch, for the 2 x 2 block inverse of A when 2N exceeds the register
// Gauss-Jordan: the block starts at `sub` (units of N^2 floats) of the vesicle's scratch, rows are
// `ld` N floats apart (1: a contiguous N x N matrix, 2: a block of a 2N x 2N matrix), and (bi, bj)
// selects the block in units of N.
struct BlkView {
  int64_t sub;
  int ld, bi, bj;
  __device__ __forceinline__ float* at(const OpCtx& c, int v, int N, int i, int j) const {
    return c.mat32(v, N, sub) + ((int64_t)(bi * N + i) * ld + bj) * N + j;
  }
};
// C = alpha A B (+ D when hasD), all N x N views.
struct OpBlk32 {
  using T = float;
  OpCtx c; BlkView A, B, C, D; float alpha; int hasD;
  __device__ void dims(int N, int& m, int& n, int& k) const { m = N; n = N; k = N; }
  __device__ float a(int v, int N, int i, int k) const { return *A.at(c, v, N, i, k); }
  __device__ float b(int v, int N, int k, int j) const { return *B.at(c, v, N, k, j); }
  __device__ void store(int v, int N, int i, int j, float acc) const {
    *C.at(c, v, N, i, j) = hasD ? fmaf(alpha, acc, *D.at(c, v, N, i, j)) : alpha * acc;
  }
};
// dst = src for N x N views; grid (ceil(N^2 / 256), M)
__global__ void __launch_bounds__(256) k_blk_copy(OpCtx c, BlkView src, BlkView dst) {
  const int v = c.vi.vid(blockIdx.y);
  const int N = c.vi.N[v];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * N) return;
  const int i = e / N, j = e - (e / N) * N;
  *dst.at(c, v, N, i, j) = *src.at(c, v, N, i, j);
}

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // k tile

// C = A B per vesicle; grid (ceil(n/64), ceil(m/64), M), 256 threads, 4x4 outputs per thread.
// Whether k_bgemm fetches the next K chunk's operands during the current chunk's products (measured per
// operator: it helps where the operand functors are cheap; OpT32's costlier functors run faster without).
template <class Op>
struct GemmPrefetch {
  static constexpr bool value = true;
};
template <>
struct GemmPrefetch<OpT32> {
  static constexpr bool value = false;
};

// Position of tile row (column) r in a shared-memory row of the k_bgemm operand tiles: the four rows
// (columns) one thread multiplies, r, r + 16, r + 32, r + 48, sit side by side, so that one 16-byte (float)
// or two (double) shared-memory loads fetch them.
__device__ __forceinline__ int gperm(int r) { return 4 * (r & 15) + (r >> 4); }
constexpr int GPAD = 4;  // row padding: rows of GT + GPAD elements stay 16-byte aligned

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p), q1 = *reinterpret_cast<const double2*>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

template <class Op>
__global__ void __launch_bounds__(256) k_bgemm(Op op, const int* __restrict__ active) {
  using T = typename Op::T;
  __shared__ __align__(16) T As[GK][GT + GPAD];
  __shared__ __align__(16) T Bs[GK][GT + GPAD];
  const int v = op.c.vi.vid(blockIdx.z);
  if (active && !active[v]) return;
  const int N = op.c.vi.N[v];
  int m, n, K;
  op.dims(N, m, n, K);
  const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
  if (r0 >= m || c0 >= n) return;
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  // the next K chunk's operands are fetched into registers while the current one is multiplied
  constexpr int PER = GK * GT / 256;
  T ra[PER], rb[PER];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      {  // A is row-major in its k index: let consecutive threads walk k
        const int kk = e % GK, rr = e / GK;
        const int gi = r0 + rr, gk = k0 + kk;
        ra[q] = (gi < m && gk < K) ? op.a(v, N, gi, gk) : T(0);
      }
      {
        const int kk = e / GT, cc = e % GT;
        const int gj = c0 + cc, gk = k0 + kk;
        rb[q] = (gj < n && gk < K) ? op.b(v, N, gk, gj) : T(0);
      }
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = tid + 256 * q;
      As[e % GK][gperm(e / GK)] = ra[q];
      Bs[e / GT][gperm(e % GT)] = rb[q];
    }
  };
  constexpr bool PF = GemmPrefetch<Op>::value;
  if constexpr (PF) fetch(0);
  for (int k0 = 0; k0 < K; k0 += GK) {
    if constexpr (PF) {
      stash();
    } else {  // operands formed straight into shared memory
      for (int e = tid; e < GK * GT; e += 256) {
        const int kk = e % GK, rr = e / GK;
        const int gi = r0 + rr, gk = k0 + kk;
        As[kk][gperm(rr)] = (gi < m && gk < K) ? op.a(v, N, gi, gk) : T(0);
      }
      for (int e = tid; e < GK * GT; e += 256) {
        const int kk = e / GT, cc = e % GT;
        const int gj = c0 + cc, gk = k0 + kk;
        Bs[kk][gperm(cc)] = (gj < n && gk < K) ? op.b(v, N, gk, gj) : T(0);
      }
    }
    __syncthreads();
    if constexpr (PF) {
      if (k0 + GK < K) fetch(k0 + GK);
    }
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      T av[4], bv[4];
      ld4(&As[kk][4 * tr], av);  // rows tr + 16 a
      ld4(&Bs[kk][4 * tc], bv);  // columns tc + 16 b
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma_t(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = r0 + tr + 16 * a, j = c0 + tc + 16 * b;
      if (i < m && j < n) op.store(v, N, i, j, acc[a][b]);
    }
}

// Where the per-vesicle LU finds its matrix: the n x n matrix at `sub` (units of N^2 doubles) of the
// vesicle's scratch with n = dm N + extra, pivots at piv + pbase(v).
template <class E>
struct LuGeoT {
  using T = E;
  VesIndex vi;
  E* scratch;
  int64_t sub;
  int dm, extra;
  int* piv;
  int pivsub;      // >= 0: pivots at 4 off + pivsub N;  < 0: at 2 off + 2 v (correction systems)
  __device__ int vid(int b) const { return vi.vid(b); }
  __device__ int n(int v) const { return dm * vi.N[v] + extra; }
  __device__ E* A(int v) const { return scratch + vi.moff[v] + sub * (int64_t)vi.N[v] * vi.N[v]; }
  __device__ int* p(int v) const {
    return pivsub >= 0 ? piv + 4 * vi.off[v] + pivsub * vi.N[v] : piv + 2 * vi.off[v] + 2 * v;
  }
};
using LuGeo = LuGeoT<double>;
using LuGeo32 = LuGeoT<float>;

// In-place LU with partial pivoting (first maximum |a| wins) of an n x n row-major matrix, n <= 2 NMAX + 8.
// Pivot k swaps rows k and piv[k]. One CTA per vesicle.
template <class Geo>
__device__ void lu_factor(typename Geo::T* A, int n, int* p, unsigned* err) {
  using E = typename Geo::T;
  __shared__ E colk[2 * NMAX + 8], rowk[2 * NMAX + 8];
  __shared__ E rv[8];
  __shared__ int ri[8];
  __shared__ int sp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k < n; ++k) {
    // pivot search in the matrix's own precision (FP64 compares are slow on this part)
    E best = E(-1);
    int idx = n;
    for (int r = k + tid; r < n; r += blockDim.x) {
      const E a = fabs(A[(int64_t)r * n + k]);
      if (a > best) { best = a; idx = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const E ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = idx; }
    __syncthreads();
    if (tid == 0) {
      E b = rv[0];
      int id = ri[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < id)) { b = rv[w]; id = ri[w]; }
      if (!(b > E(0))) { atomicOr(err, ERR_PIVOT); id = k; }
      sp = id;
      p[k] = id;
    }
    __syncthreads();
    const int pr = sp;
    if (pr != k) {
      for (int j = tid; j < n; j += blockDim.x) {
        const E t = A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = A[(int64_t)pr * n + j];
        A[(int64_t)pr * n + j] = t;
      }
      __syncthreads();
    }
    const E piv_v = A[(int64_t)k * n + k];
    const E inv = (piv_v != E(0)) ? E(1) / piv_v : E(0);
    for (int j = k + 1 + tid; j < n; j += blockDim.x) rowk[j] = A[(int64_t)k * n + j];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
      const E l = A[(int64_t)i * n + k] * inv;
      A[(int64_t)i * n + k] = l;
      colk[i] = l;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int i = k + 1 + wid; i < n; i += nw) {  // rows by warps, columns by lanes
      const E li = colk[i];
      E* Ai = A + (int64_t)i * n;
      for (int j = k + 1 + lane; j < n; j += 32) Ai[j] = fma_t(-li, rowk[j], Ai[j]);
    }
    __syncthreads();
  }
}

template <class Geo>
__global__ void __launch_bounds__(256) k_lu(Geo geo, unsigned* err, const int* __restrict__ active) {
  const int v = geo.vid(blockIdx.x);
  if (active && !active[v]) return;
  lu_factor<Geo>(geo.A(v), geo.n(v), geo.p(v), err);
}

// The same factorisation staged through shared memory (dynamic, n^2 elements): for matrices that
// fit, the elimination's many passes over the trailing block stay on chip.
template <class Geo>
__global__ void __launch_bounds__(256) k_lu_smem(Geo geo, unsigned* err, const int* __restrict__ active) {
  using E = typename Geo::T;
  extern __shared__ unsigned char lu_raw[];
  E* As = reinterpret_cast<E*>(lu_raw);
  const int v = geo.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int n = geo.n(v);
  E* A = geo.A(v);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) As[e] = A[e];
  __syncthreads();
  lu_factor<Geo>(As, n, geo.p(v), err);
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) A[e] = As[e];
}

// Reciprocal of a Gauss-Jordan pivot: the hardware approximation (rcp.approx, within one unit in the last
// place); the FP32 inverses only precondition refinement, and the IEEE division's longer sequence sat on
// the critical path of every elimination step.
__device__ __forceinline__ float gj_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// In-place FP32 inverse of the n x n matrix at geo (n <= 16 RA = TC RB) by Gauss-Jordan exchange steps
// with partial pivoting: step k takes as pivot p the row not yet used with the largest |T[p][k]| (first
// wins) and exchanges equation p with unknown k,
//   T[p][k] <- 1/t,  T[p][j] <- -T[p][j]/t,  T[i][k] <- T[i][k]/t,  T[i][j] <- T[i][j] - T[i][k] T[p][j]/t
// (t = T[p][k]). After n steps row i expresses unknown step(i) through the right-hand-side entries
// pivot(j) of the columns, so inv[step(i)][pivot(j)] = T[i][j]; no rows move.
// 16 TC threads form a 16 x TC grid, thread (tr, tc) = (tid % 16, tid / 16) keeping T[tr + 16a][tc + TC b]
// (a < RA, b < RB) in registers as pairs over b for the paired FP32 update. The column of step k sits in
// register b = k / TC of the half-warp tc = k % TC, which also finds the pivot by shuffles; column k and
// row p are broadcast through shared memory laid out per owner ([tr][a] and [tc][b]) so that each thread
// reads its values as vectors. Two barriers a step.
// The elimination as a device function of the whole CTA (16 TC threads): src and dst (global or shared
// memory, row-major n x n, possibly the same) are read before and written after the elimination.
template <int RA, int RB, int TC>
__device__ void gj_invert(const float* src, float* dst, int n, unsigned* err) {
  static_assert(RB % 2 == 0 && RA % 2 == 0 && RA <= 8 && 16 * RA == TC * RB, "square grid of pairs");
  constexpr int NP = 16 * RA, H = RB / 2;
  __shared__ __align__(16) float colb[2][NP], rowb[2][NP];  // colb[tr * RA + a], rowb[tc * RB + b]
  __shared__ int psel[2], pk[NP], rstep[NP];
  const float* A = src;
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  float2 T[RA][H];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      T[a][h].x = (i < n && j0 < n) ? A[(int64_t)i * n + j0] : 0.f;
      T[a][h].y = (i < n && j1 < n) ? A[(int64_t)i * n + j1] : 0.f;
    }
  for (int e = tid; e < 2 * NP; e += blockDim.x) {
    (&colb[0][0])[e] = 0.f;
    (&rowb[0][0])[e] = 0.f;
  }
  __syncthreads();
  unsigned used = 0u;  // bit a: row tr + 16 a has been a pivot
  bool bad = false;
  const unsigned half = (tc & 1) ? 0xffff0000u : 0x0000ffffu;
#pragma unroll
  for (int kb = 0; kb < RB; ++kb) {
    for (int kc = 0; kc < TC; ++kc) {
      const int k = TC * kb + kc;
      if (k >= n) break;
      const int buf = k & 1;  // double-buffered broadcasts: two barriers per step suffice
      if (tc == kc) {         // the half-warp holding column k: publish it and find the pivot
        float best = -1.f;
        int bi = NP;
        float cv[RA];
#pragma unroll
        for (int a = 0; a < RA; ++a) {
          const int i = tr + 16 * a;
          cv[a] = (kb & 1) ? T[a][kb >> 1].y : T[a][kb >> 1].x;
          // the first unused row is always a candidate, so a NaN column still yields a row
          if (i < n && !((used >> a) & 1u) && (fabsf(cv[a]) > best || bi == NP)) { best = fabsf(cv[a]); bi = i; }
        }
        if constexpr (RA >= 4) {
#pragma unroll
          for (int a = 0; a < RA; a += 4)
            *reinterpret_cast<float4*>(&colb[buf][tr * RA + a]) = make_float4(cv[a], cv[a + 1], cv[a + 2], cv[a + 3]);
        } else {
          *reinterpret_cast<float2*>(&colb[buf][tr * RA]) = make_float2(cv[0], cv[1]);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          const float ob = __shfl_xor_sync(half, best, o);
          const int oi = __shfl_xor_sync(half, bi, o);
          if (oi < NP && (bi == NP || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
        }
        if (tr == 0) psel[buf] = (bi < n && best > 0.f) ? bi : -1 - (bi < n ? bi : n - 1);
      }
      __syncthreads();
      int p = psel[buf];
      if (p < 0) { bad = true; p = -1 - p; }  // zero or NaN pivot column
      const int pr = p & 15, pa = p >> 4;
      if (tr == pr) {  // owners of row p publish it
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
            if constexpr (H == 1) {
              *reinterpret_cast<float2*>(&rowb[buf][tc * RB]) = T[a][0];
            } else {
#pragma unroll
              for (int h = 0; h < H; h += 2)
                *reinterpret_cast<float4*>(&rowb[buf][tc * RB + 2 * h]) =
                    make_float4(T[a][h].x, T[a][h].y, T[a][h + 1].x, T[a][h + 1].y);
            }
            used |= 1u << a;
          }
      }
      if (tid == 0) { pk[k] = p; rstep[p] = k; }
      __syncthreads();
      float pv = colb[buf][pr * RA + pa];
      if (bad || !(pv != 0.f)) { bad = true; pv = 1.f; }
      const float ip = gj_rcp(pv);
      float c[RA];
      float2 u[H];
      if constexpr (RA >= 4) {
#pragma unroll
        for (int a = 0; a < RA; a += 4) {
          const float4 w = *reinterpret_cast<const float4*>(&colb[buf][tr * RA + a]);
          c[a] = w.x; c[a + 1] = w.y; c[a + 2] = w.z; c[a + 3] = w.w;
        }
      } else {
        const float2 w = *reinterpret_cast<const float2*>(&colb[buf][tr * RA]);
        c[0] = w.x; c[1] = w.y;
      }
#pragma unroll
      for (int h = 0; h < H; ++h) u[h] = __fmul2_rn(*reinterpret_cast<const float2*>(&rowb[buf][tc * RB + 2 * h]), make_float2(ip, ip));
      if (tc == kc) {  // column k itself: T[i][k] <- T[i][k] / t
        if (kb & 1) u[kb >> 1].y = 1.f - ip; else u[kb >> 1].x = 1.f - ip;
      }
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int h = 0; h < H; ++h) T[a][h] = __ffma2_rn(make_float2(-c[a], -c[a]), u[h], T[a][h]);
      if (tr == pr) {  // row p: T[p][j] <- -T[p][j] / t, T[p][k] <- 1 / t
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
#pragma unroll
            for (int h = 0; h < H; ++h) T[a][h] = make_float2(-u[h].x, -u[h].y);
            if (tc == kc) {
              if (kb & 1) T[a][kb >> 1].y = ip; else T[a][kb >> 1].x = ip;
            }
          }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      if (i < n && j0 < n) dst[(int64_t)rstep[i] * n + pk[j0]] = T[a][h].x;
      if (i < n && j1 < n) dst[(int64_t)rstep[i] * n + pk[j1]] = T[a][h].y;
    }
  if (bad && tid == 0) atomicOr(err, ERR_PIVOT);
  __syncthreads();
}

// The same exchange steps without pivoting: step k takes row k, so the row and the column of a step are
// known in advance and their owners publish both before a single barrier (one barrier a step instead of
// two, and no pivot search). A pivot with |t| <= GJ_NP_TOL max|A| ends the attempt: it returns false and
// writes nothing (uniformly across the CTA), and the caller runs the pivoting elimination. Otherwise the
// result is the inverse in place (inv[i][j] = T[i][j], no permutation).
constexpr float GJ_NP_TOL = 1e-4f;

template <int RA, int RB, int TC>
__device__ bool gj_invert_np(const float* src, float* dst, int n) {
  static_assert(RB % 2 == 0 && RA % 2 == 0 && RA <= 8 && 16 * RA == TC * RB, "square grid of pairs");
  constexpr int NP = 16 * RA, H = RB / 2, NW = 16 * TC / 32;
  __shared__ __align__(16) float colb[2][NP], rowb[2][NP];
  __shared__ float wmax[NW];
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  float2 T[RA][H];
  float mx = 0.f;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      T[a][h].x = (i < n && j0 < n) ? src[(int64_t)i * n + j0] : 0.f;
      T[a][h].y = (i < n && j1 < n) ? src[(int64_t)i * n + j1] : 0.f;
      mx = fmaxf(mx, fmaxf(fabsf(T[a][h].x), fabsf(T[a][h].y)));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  mx = wmax[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) mx = fmaxf(mx, wmax[w]);
  const float thr = GJ_NP_TOL * mx;
  bool ok = mx > 0.f;
#pragma unroll
  for (int kb = 0; kb < RB; ++kb) {
#pragma unroll 1
    for (int kc = 0; kc < TC; ++kc) {
      const int k = TC * kb + kc;
      if (k >= n) break;
      const int buf = k & 1;
      const int pr = k & 15, pa = k >> 4;
      if (tc == kc) {  // column k
        float cv[RA];
#pragma unroll
        for (int a = 0; a < RA; ++a) cv[a] = (kb & 1) ? T[a][kb >> 1].y : T[a][kb >> 1].x;
        if constexpr (RA >= 4) {
#pragma unroll
          for (int a = 0; a < RA; a += 4)
            *reinterpret_cast<float4*>(&colb[buf][tr * RA + a]) = make_float4(cv[a], cv[a + 1], cv[a + 2], cv[a + 3]);
        } else {
          *reinterpret_cast<float2*>(&colb[buf][tr * RA]) = make_float2(cv[0], cv[1]);
        }
      }
      if (tr == pr) {  // row k
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
            if constexpr (H == 1) {
              *reinterpret_cast<float2*>(&rowb[buf][tc * RB]) = T[a][0];
            } else {
#pragma unroll
              for (int h = 0; h < H; h += 2)
                *reinterpret_cast<float4*>(&rowb[buf][tc * RB + 2 * h]) =
                    make_float4(T[a][h].x, T[a][h].y, T[a][h + 1].x, T[a][h + 1].y);
            }
          }
      }
      __syncthreads();
      float pv = colb[buf][pr * RA + pa];
      if (!(fabsf(pv) > thr)) { ok = false; pv = 1.f; }
      const float ip = gj_rcp(pv);
      float c[RA];
      float2 u[H];
      if constexpr (RA >= 4) {
#pragma unroll
        for (int a = 0; a < RA; a += 4) {
          const float4 w = *reinterpret_cast<const float4*>(&colb[buf][tr * RA + a]);
          c[a] = w.x; c[a + 1] = w.y; c[a + 2] = w.z; c[a + 3] = w.w;
        }
      } else {
        const float2 w = *reinterpret_cast<const float2*>(&colb[buf][tr * RA]);
        c[0] = w.x; c[1] = w.y;
      }
#pragma unroll
      for (int h = 0; h < H; ++h) u[h] = __fmul2_rn(*reinterpret_cast<const float2*>(&rowb[buf][tc * RB + 2 * h]), make_float2(ip, ip));
      if (tc == kc) {
        if (kb & 1) u[kb >> 1].y = 1.f - ip; else u[kb >> 1].x = 1.f - ip;
      }
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int h = 0; h < H; ++h) T[a][h] = __ffma2_rn(make_float2(-c[a], -c[a]), u[h], T[a][h]);
      if (tr == pr) {
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
#pragma unroll
            for (int h = 0; h < H; ++h) T[a][h] = make_float2(-u[h].x, -u[h].y);
            if (tc == kc) {
              if (kb & 1) T[a][kb >> 1].y = ip; else T[a][kb >> 1].x = ip;
            }
          }
      }
    }
  }
  // every thread took the same decisions from the same shared values; the barrier also ends the reads
  // of src before dst (possibly the same memory) is written
  __syncthreads();
  if (!ok) return false;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      if (i < n && j0 < n) dst[(int64_t)i * n + j0] = T[a][h].x;
      if (i < n && j1 < n) dst[(int64_t)i * n + j1] = T[a][h].y;
    }
  __syncthreads();
  return true;
}

// The same elimination two exchange steps per barrier (n even): the owners of columns k, k + 1 and rows k, k + 1
// publish them before one barrier, and every thread applies both steps to its entries at once, step k + 1's
// pivot row and column taken as step k leaves them (computed locally from the four published vectors), so the
// result is that of the two single steps. The pivots P00 and P11 - P10 P01 / P00 are held to the same
// threshold (GJ_NP_TOL max|A|); a smaller one ends the attempt as in gj_invert_np. Half the barriers of
// gj_invert_np, whose steps are bound by the barrier and the pivot's latency rather than by the FP32 work.
template <int RA, int RB, int TC>
__device__ bool gj_invert_np2(const float* src, float* dst, int n) {
  static_assert(RB % 2 == 0 && RA % 2 == 0 && RA <= 8 && 16 * RA == TC * RB && TC % 2 == 0, "square grid of pairs");
  constexpr int NP = 16 * RA, H = RB / 2, NW = 16 * TC / 32;
  __shared__ __align__(16) float colb[2][2][NP], rowb[2][2][NP];
  __shared__ float wmax[NW];
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  float2 T[RA][H];
  float mx = 0.f;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      T[a][h].x = (i < n && j0 < n) ? src[(int64_t)i * n + j0] : 0.f;
      T[a][h].y = (i < n && j1 < n) ? src[(int64_t)i * n + j1] : 0.f;
      mx = fmaxf(mx, fmaxf(fabsf(T[a][h].x), fabsf(T[a][h].y)));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((tid & 31) == 0) wmax[tid >> 5] = mx;
  __syncthreads();
  mx = wmax[0];
#pragma unroll
  for (int w = 1; w < NW; ++w) mx = fmaxf(mx, wmax[w]);
  const float thr = GJ_NP_TOL * mx;
  bool ok = mx > 0.f;
#pragma unroll
  for (int kb = 0; kb < RB; ++kb) {
#pragma unroll 1
    for (int kc = 0; kc < TC; kc += 2) {
      const int k = TC * kb + kc;  // even: rows k, k + 1 share a (pa), columns k, k + 1 share b (kb)
      if (k >= n) break;
      const int buf = (k >> 1) & 1;
      const int pr = k & 15, pa = k >> 4;
      if (tc == kc || tc == kc + 1) {  // column k or k + 1
        float* cb = colb[buf][tc - kc];
        float cv[RA];
#pragma unroll
        for (int a = 0; a < RA; ++a) cv[a] = (kb & 1) ? T[a][kb >> 1].y : T[a][kb >> 1].x;
        if constexpr (RA >= 4) {
#pragma unroll
          for (int a = 0; a < RA; a += 4)
            *reinterpret_cast<float4*>(&cb[tr * RA + a]) = make_float4(cv[a], cv[a + 1], cv[a + 2], cv[a + 3]);
        } else {
          *reinterpret_cast<float2*>(&cb[tr * RA]) = make_float2(cv[0], cv[1]);
        }
      }
      if (tr == pr || tr == pr + 1) {  // row k or k + 1
        float* rb = rowb[buf][tr - pr];
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
            if constexpr (H == 1) {
              *reinterpret_cast<float2*>(&rb[tc * RB]) = T[a][0];
            } else {
#pragma unroll
              for (int h = 0; h < H; h += 2)
                *reinterpret_cast<float4*>(&rb[tc * RB + 2 * h]) =
                    make_float4(T[a][h].x, T[a][h].y, T[a][h + 1].x, T[a][h + 1].y);
            }
          }
      }
      __syncthreads();
      const float p00 = colb[buf][0][pr * RA + pa], p10 = colb[buf][0][(pr + 1) * RA + pa];
      const float p01 = colb[buf][1][pr * RA + pa], p11 = colb[buf][1][(pr + 1) * RA + pa];
      float t1 = p00;
      if (!(fabsf(t1) > thr)) { ok = false; t1 = 1.f; }
      const float i1 = gj_rcp(t1);
      const float a01 = p01 * i1, a10 = p10 * i1;
      float t2 = fmaf(-a10, p01, p11);  // the pivot of step k + 1 after step k
      if (!(fabsf(t2) > thr)) { ok = false; t2 = 1.f; }
      const float i2 = gj_rcp(t2);
      // the two steps in their sequential form: column k + 1 and row k + 1 as step k leaves them,
      //   c1'_i = c1_i - c0_i p01 / p00,  r1'_j = r1_j - p10 r0_j / p00,
      // then T_ij -= c0_i r0_j / p00 + c1'_i r1'_j / t2 (the block inverse's explicit form would amplify
      // rounding by |P| / t2 where the second pivot is small)
      float c0[RA], c1[RA];
      if constexpr (RA >= 4) {
#pragma unroll
        for (int a = 0; a < RA; a += 4) {
          const float4 w0 = *reinterpret_cast<const float4*>(&colb[buf][0][tr * RA + a]);
          const float4 w1 = *reinterpret_cast<const float4*>(&colb[buf][1][tr * RA + a]);
          c0[a] = w0.x; c0[a + 1] = w0.y; c0[a + 2] = w0.z; c0[a + 3] = w0.w;
          c1[a] = w1.x; c1[a + 1] = w1.y; c1[a + 2] = w1.z; c1[a + 3] = w1.w;
        }
      } else {
        const float2 w0 = *reinterpret_cast<const float2*>(&colb[buf][0][tr * RA]);
        const float2 w1 = *reinterpret_cast<const float2*>(&colb[buf][1][tr * RA]);
        c0[0] = w0.x; c0[1] = w0.y;
        c1[0] = w1.x; c1[1] = w1.y;
      }
#pragma unroll
      for (int a = 0; a < RA; ++a) c1[a] = (tr == pr && a == pa) ? -a01 : fmaf(-c0[a], a01, c1[a]);
      float2 u0[H], u1[H];
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const float2 r0 = *reinterpret_cast<const float2*>(&rowb[buf][0][tc * RB + 2 * h]);
        const float2 r1 = *reinterpret_cast<const float2*>(&rowb[buf][1][tc * RB + 2 * h]);
        u0[h] = __fmul2_rn(make_float2(i1, i1), r0);
        u1[h] = __fmul2_rn(make_float2(i2, i2), __ffma2_rn(make_float2(-a10, -a10), r0, r1));
      }
      // columns k, k + 1 through the same update: (u0, u1) there = (1 - i1, a10 i2) and (a01, 1 - i2)
      const bool ck = tc == kc, ck1 = tc == kc + 1;
      float2 m0 = u0[kb >> 1], m1 = u1[kb >> 1];
      if (ck || ck1) {
        const float v0 = ck ? 1.f - i1 : a01, v1 = ck ? a10 * i2 : 1.f - i2;
        if (kb & 1) { m0.y = v0; m1.y = v1; } else { m0.x = v0; m1.x = v1; }
      }
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int h = 0; h < H; ++h) {
          const float2 e0 = (h == (kb >> 1)) ? m0 : u0[h], e1 = (h == (kb >> 1)) ? m1 : u1[h];
          T[a][h] = __ffma2_rn(make_float2(-c0[a], -c0[a]), e0, T[a][h]);
          T[a][h] = __ffma2_rn(make_float2(-c1[a], -c1[a]), e1, T[a][h]);
        }
      if (tr == pr || tr == pr + 1) {  // rows k, k + 1 as the two exchange steps leave them
        const bool second = tr != pr;
#pragma unroll
        for (int a = 0; a < RA; ++a)
          if (a == pa) {
#pragma unroll
            for (int h = 0; h < H; ++h)
              T[a][h] = second ? make_float2(-u1[h].x, -u1[h].y)
                               : __ffma2_rn(make_float2(a01, a01), u1[h], make_float2(-u0[h].x, -u0[h].y));
            if (ck || ck1) {
              const float qv = second ? (ck ? -a10 * i2 : i2) : (ck ? fmaf(a01 * a10, i2, i1) : -a01 * i2);
              if (kb & 1) T[a][kb >> 1].y = qv; else T[a][kb >> 1].x = qv;
            }
          }
      }
    }
  }
  __syncthreads();
  if (!ok) return false;
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const int i = tr + 16 * a, j0 = tc + 2 * TC * h, j1 = j0 + TC;
      if (i < n && j0 < n) dst[(int64_t)i * n + j0] = T[a][h].x;
      if (i < n && j1 < n) dst[(int64_t)i * n + j1] = T[a][h].y;
    }
  __syncthreads();
  return true;
}

// A dense batch of n x n row-major FP32 matrices, matrix v at base + v n^2.
struct DenseGeo32 {
  float* base;
  int nn;
  __device__ int vid(int b) const { return b; }
  __device__ int n(int) const { return nn; }
  __device__ float* A(int v) const { return base + (int64_t)v * nn * nn; }
};

// CTAs per SM the register allocation must allow: 128-thread shapes (64 x 64 matrices) 5, else 2.
#define GJ_MIN_CTAS(TC) ((TC) == 8 ? 5 : 2)

// In-place inverse of matrix blockIdx.x of geo; fallbacks (may be null) counts the matrices that needed
// the pivoting elimination.
template <int RA, int RB, int TC, class Geo>
__global__ void __launch_bounds__(16 * TC, GJ_MIN_CTAS(TC)) k_gj_inverse(Geo geo, unsigned* err, const int* __restrict__ active,
                                                           int* fallbacks) {
  const int v = geo.vid(blockIdx.x);
  if (active && !active[v]) return;
  float* A = geo.A(v);
  const int n = geo.n(v);
  if (!((n % 2 == 0) ? gj_invert_np2<RA, RB, TC>(A, A, n) : gj_invert_np<RA, RB, TC>(A, A, n))) {
    if (fallbacks && threadIdx.x == 0) atomicAdd(fallbacks, 1);
    gj_invert<RA, RB, TC>(A, A, geo.n(v), err);
  }
}

// Solve LU x = b in place for one vector b in shared memory (length n); warp 0 works, the
// block synchronises on exit. Row-oriented substitution with warp dot products.
template <class F>
__device__ void lu_solve_vec(const F* LU, const int* p, int n, double* b) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    if (lane == 0)
      for (int k = 0; k < n; ++k) {
        const int q = p[k];
        if (q != k) { const double t = b[k]; b[k] = b[q]; b[q] = t; }
      }
    __syncwarp();
    for (int i = 1; i < n; ++i) {
      double s = 0.0;
      for (int k = lane; k < i; k += 32) s = fma((double)LU[(int64_t)i * n + k], b[k], s);
      s = warp_sum(s);
      if (lane == 0) b[i] -= s;
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k < n; k += 32) s = fma((double)LU[(int64_t)i * n + k], b[k], s);
      s = warp_sum(s);
      if (lane == 0) b[i] = (b[i] - s) / (double)LU[(int64_t)i * n + i];
      __syncwarp();
    }
  }
  __syncthreads();
}

// W <- L^{-1} W for the N x 2N block W using the LU of L at slot s; thread per column.
template <class E>
__global__ void __launch_bounds__(256) k_lu_solve_cols(VesIndex vi, E* scratch, int s,
                                                       const int* piv, const int* __restrict__ active) {
  const int v = vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int nc = 2 * N;
  const int col = threadIdx.x;
  if (col >= nc) return;
  const E* LU = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::L) * (int64_t)N * N;
  E* W = scratch + vi.moff[v] + MatLayout::W * (int64_t)N * N;
  const int* p = piv + 4 * vi.off[v] + s * N;
  for (int k = 0; k < N; ++k) {
    const int q = p[k];
    if (q != k) {
      const E t = W[(int64_t)k * nc + col];
      W[(int64_t)k * nc + col] = W[(int64_t)q * nc + col];
      W[(int64_t)q * nc + col] = t;
    }
  }
  for (int i = 1; i < N; ++i) {
    E s2 = W[(int64_t)i * nc + col];
    for (int k = 0; k < i; ++k) s2 = fma_t(-LU[(int64_t)i * N + k], W[(int64_t)k * nc + col], s2);
    W[(int64_t)i * nc + col] = s2;
  }
  for (int i = N - 1; i >= 0; --i) {
    E s2 = W[(int64_t)i * nc + col];
    for (int k = i + 1; k < N; ++k) s2 = fma_t(-LU[(int64_t)i * N + k], W[(int64_t)k * nc + col], s2);
    W[(int64_t)i * nc + col] = s2 / LU[(int64_t)i * N + i];
  }
}

}  // namespace vs
