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
  __device__ __forceinline__ double* mat(int v, int N, int64_t sub) const {
    return scratch + vi.moff[v] + sub * (int64_t)N * N;
  }
  __device__ __forceinline__ double dcirc(int v, int N, int m) const {
    m %= N;
    if (m < 0) m += N;
    return tab[vi.toff[v] + m];
  }
};

// T = S Ten at slot s.
struct OpT {
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

constexpr int GT = 64;   // output tile
constexpr int GK = 16;   // k tile

// C = A B per vesicle; grid (ceil(n/64), ceil(m/64), M), 256 threads, 4x4 outputs per thread.
template <class Op>
__global__ void __launch_bounds__(256) k_bgemm(Op op, const int* __restrict__ active) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int v = blockIdx.z;
  if (active && !active[v]) return;
  const int N = op.c.vi.N[v];
  int m, n, K;
  op.dims(N, m, n, K);
  const int r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
  if (r0 >= m || c0 >= n) return;
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = tid; e < GK * GT; e += 256) {
      // A is row-major in its k index: let consecutive threads walk k
      const int kk = e % GK, rr = e / GK;
      const int gi = r0 + rr, gk = k0 + kk;
      As[kk][rr] = (gi < m && gk < K) ? op.a(v, N, gi, gk) : 0.0;
    }
    for (int e = tid; e < GK * GT; e += 256) {
      const int kk = e / GT, cc = e % GT;
      const int gj = c0 + cc, gk = k0 + kk;
      Bs[kk][cc] = (gj < n && gk < K) ? op.b(v, N, gk, gj) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tr + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tc + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
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
struct LuGeo {
  VesIndex vi;
  double* scratch;
  int64_t sub;
  int dm, extra;
  int* piv;
  int pivsub;      // >= 0: pivots at 4 off + pivsub N;  < 0: at 2 off + 2 v (correction systems)
  __device__ int n(int v) const { return dm * vi.N[v] + extra; }
  __device__ double* A(int v) const { return scratch + vi.moff[v] + sub * (int64_t)vi.N[v] * vi.N[v]; }
  __device__ int* p(int v) const {
    return pivsub >= 0 ? piv + 4 * vi.off[v] + pivsub * vi.N[v] : piv + 2 * vi.off[v] + 2 * v;
  }
};

// In-place LU with partial pivoting (first maximum |a| wins) of an n x n row-major matrix, n <= 2 NMAX + 8.
// Pivot k swaps rows k and piv[k]. One CTA per vesicle.
__global__ void __launch_bounds__(256) k_lu(LuGeo geo, unsigned* err, const int* __restrict__ active) {
  __shared__ double colk[2 * NMAX + 8], rowk[2 * NMAX + 8];
  __shared__ double rv[8];
  __shared__ int ri[8];
  __shared__ int sp;
  const int v = blockIdx.x;
  if (active && !active[v]) return;
  const int n = geo.n(v);
  double* A = geo.A(v);
  int* p = geo.p(v);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k < n; ++k) {
    double best = -1.0;
    int idx = n;
    for (int r = k + tid; r < n; r += blockDim.x) {
      const double a = fabs(A[(int64_t)r * n + k]);
      if (a > best) { best = a; idx = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
    }
    if (lane == 0) { rv[wid] = best; ri[wid] = idx; }
    __syncthreads();
    if (tid == 0) {
      double b = rv[0];
      int id = ri[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (rv[w] > b || (rv[w] == b && ri[w] < id)) { b = rv[w]; id = ri[w]; }
      if (!(b > 0.0)) { atomicOr(err, ERR_PIVOT); id = k; }
      sp = id;
      p[k] = id;
    }
    __syncthreads();
    const int pr = sp;
    if (pr != k) {
      for (int j = tid; j < n; j += blockDim.x) {
        const double t = A[(int64_t)k * n + j];
        A[(int64_t)k * n + j] = A[(int64_t)pr * n + j];
        A[(int64_t)pr * n + j] = t;
      }
      __syncthreads();
    }
    const double piv_v = A[(int64_t)k * n + k];
    const double inv = (piv_v != 0.0) ? 1.0 / piv_v : 0.0;
    for (int j = k + 1 + tid; j < n; j += blockDim.x) rowk[j] = A[(int64_t)k * n + j];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) {
      const double l = A[(int64_t)i * n + k] * inv;
      A[(int64_t)i * n + k] = l;
      colk[i] = l;
    }
    __syncthreads();
    const int rem = n - k - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, j = k + 1 + e % rem;
      A[(int64_t)i * n + j] = fma(-colk[i], rowk[j], A[(int64_t)i * n + j]);
    }
    __syncthreads();
  }
}

// Solve LU x = b in place for one vector b in shared memory (length n); warp 0 works, the
// block synchronises on exit. Row-oriented substitution with warp dot products.
__device__ void lu_solve_vec(const double* LU, const int* p, int n, double* b) {
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
      for (int k = lane; k < i; k += 32) s = fma(LU[(int64_t)i * n + k], b[k], s);
      s = warp_sum(s);
      if (lane == 0) b[i] -= s;
      __syncwarp();
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1 + lane; k < n; k += 32) s = fma(LU[(int64_t)i * n + k], b[k], s);
      s = warp_sum(s);
      if (lane == 0) b[i] = (b[i] - s) / LU[(int64_t)i * n + i];
      __syncwarp();
    }
  }
  __syncthreads();
}

// W <- L^{-1} W for the N x 2N block W using the LU of L at slot s; thread per column.
__global__ void __launch_bounds__(256) k_lu_solve_cols(VesIndex vi, double* scratch, int s,
                                                       const int* piv, const int* __restrict__ active) {
  const int v = blockIdx.x;
  if (active && !active[v]) return;
  const int N = vi.N[v];
  const int nc = 2 * N;
  const int col = threadIdx.x;
  if (col >= nc) return;
  const double* LU = scratch + vi.moff[v] + (MatLayout::slot(s) + MatLayout::L) * (int64_t)N * N;
  double* W = scratch + vi.moff[v] + MatLayout::W * (int64_t)N * N;
  const int* p = piv + 4 * vi.off[v] + s * N;
  for (int k = 0; k < N; ++k) {
    const int q = p[k];
    if (q != k) {
      const double t = W[(int64_t)k * nc + col];
      W[(int64_t)k * nc + col] = W[(int64_t)q * nc + col];
      W[(int64_t)q * nc + col] = t;
    }
  }
  for (int i = 1; i < N; ++i) {
    double s2 = W[(int64_t)i * nc + col];
    for (int k = 0; k < i; ++k) s2 = fma(-LU[(int64_t)i * N + k], W[(int64_t)k * nc + col], s2);
    W[(int64_t)i * nc + col] = s2;
  }
  for (int i = N - 1; i >= 0; --i) {
    double s2 = W[(int64_t)i * nc + col];
    for (int k = i + 1; k < N; ++k) s2 = fma(-LU[(int64_t)i * N + k], W[(int64_t)k * nc + col], s2);
    W[(int64_t)i * nc + col] = s2 / LU[(int64_t)i * N + i];
  }
}

}  // namespace vs
