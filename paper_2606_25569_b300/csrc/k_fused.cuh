// Fused per-vesicle FP32 operator products of the mixed-precision path, for vesicles of at most 64 points.
//
// The refinement of every per-vesicle solve (Sec. 3.1 operators; advection, relaxation and tension steps)
// is preconditioned by FP32 copies of T = S Ten and L = P T (Eqs. bending_op .. PTop) and, for the
// relaxation (Eq. relaxation_disc), of W = L^{-1} P B and A = I - dt (B - T W) with B = -kappa S
// blockdiag(D4, D4), D4 = (D_s D_s)(D_s D_s); k_dense.cuh states the products (OpT32 .. OpA32). Formed by one
// batched GEMM launch per product, every intermediate goes through device memory (hundreds of MB at
// thousands of vesicles, far beyond L2). Here one CTA per vesicle forms a whole chain in shared memory:
//   k_fused_tl     T and L of an operator slot (L then inverted in place by k_gj_inverse);
//   k_fused_relax  W and A from S, T and L^{-1} of the slot (A then inverted in place by k_gj_inverse).
// The 2N-row matrices are taken one row block (the x or the y rows) at a time, and every N x N block is
// embedded in a 64 x 64 block padded with zeros (the x columns of a 2N-column matrix at 0.., the y columns at
// 64..), so every product is a 64 x 64 by 64 x (64 or 128) product and the padding contributes nothing: the
// entries written back are those of the unpadded products. The products run as register-tiled FP32 GEMMs
// from shared memory (fz_gemm), two CTAs per SM; their sums run in another order than k_bgemm's, so the two
// agree to FP32 rounding, which is all a preconditioner of FP64 refinement needs.
#pragma once
#include "k_dense.cuh"

namespace vs {

constexpr int FZ = 64;              // embedded block order
constexpr int FL1 = FZ + 4;         // leading dimension (floats) of 64-column shared arrays (rows 16-byte aligned)
constexpr int FL2 = 2 * FZ + 4;     // of 128-column shared arrays
constexpr int FUSED_THREADS = 256;  // 8 warps: thread (tr, tc) = (warp, lane)

// acc[a][b] += sum_{k < K} A[8 tr + a][k] B[k][NB tc + b] (K a multiple of 4): both operands row-major in shared
// memory (leading dimensions lda, ldb multiples of 4), a 64 x 32 NB block of outputs over the CTA. A warp shares
// its rows, so its A loads (four k at a time) are broadcasts and its B loads one contiguous run.
template <int NB>
__device__ __forceinline__ void fz_gemm(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
                                        int K, float (&acc)[8][NB]) {
  static_assert(NB == 2 || NB == 4, "tile shape");
  const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
  const float* a = A + 8 * tr * lda;
  const float* b = B + NB * tc;
#pragma unroll 2
  for (int k0 = 0; k0 < K; k0 += 4) {
    float4 av[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) av[i] = *reinterpret_cast<const float4*>(a + i * lda + k0);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      float bv[NB];
      if constexpr (NB == 4) {
        const float4 t = *reinterpret_cast<const float4*>(b + (k0 + kk) * ldb);
        bv[0] = t.x; bv[1] = t.y; bv[2] = t.z; bv[3] = t.w;
      } else {
        const float2 t = *reinterpret_cast<const float2*>(b + (k0 + kk) * ldb);
        bv[0] = t.x; bv[1] = t.y;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float ai = kk == 0 ? av[i].x : kk == 1 ? av[i].y : kk == 2 ? av[i].z : av[i].w;
#pragma unroll
        for (int j = 0; j < NB; j += 2) {  // paired FP32 FMAs (each lane rounded as fmaf)
          const float2 c = __ffma2_rn(make_float2(ai, ai), make_float2(bv[j], bv[j + 1]),
                                      make_float2(acc[i][j], acc[i][j + 1]));
          acc[i][j] = c.x;
          acc[i][j + 1] = c.y;
        }
      }
    }
  }
}

template <int NB>
__device__ __forceinline__ void fz_zero(float (&acc)[8][NB]) {
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[i][j] = 0.f;
}

// Real column (or row) of embedded index c of a 2N-wide matrix (x part at 0.., y part at 64..), or -1 (padding).
__device__ __forceinline__ int fz_real(int c, int N) { return c < FZ ? (c < N ? c : -1) : (c - FZ < N ? c - FZ + N : -1); }

// D_s = diag(1/|X_alpha|) D_alpha of vesicle v into Ds (row-major, ld FL1), zero outside N x N; the tangent
// components x_s, y_s of its points into txs, tys (zero past N).
__device__ void fz_load_ds(const OpCtx& c, int v, int N, float* Ds, float* txs, float* tys) {
  const int64_t o = c.vi.off[v];
  for (int e = threadIdx.x; e < FZ * FZ; e += blockDim.x) {
    const int i = e >> 6, k = e & (FZ - 1);
    Ds[i * FL1 + k] = (i < N && k < N) ? c.dcirc32(v, N, i - k) * c.g32[o + i].x : 0.f;
  }
  for (int i = threadIdx.x; i < FZ; i += blockDim.x) {
    const float4 g = (i < N) ? c.g32[o + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    txs[i] = g.y;
    tys[i] = g.z;
  }
}

// Asynchronous copies into shared memory (cp.async, 8 bytes; a source size of 0 fills zeros).
__device__ __forceinline__ void fz_cp8(float* dst, const float* src, bool real) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(real ? 8 : 0) : "memory");
}
__device__ __forceinline__ void fz_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void fz_cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// Rows r0 .. r0 + N - 1 of a row-major matrix in device memory with nb = 1 or 2 column blocks of N columns
// (leading dimension nb N) into X[i][64 b + k] (ld ldx), zero over the rest of the 64 x 64 nb region, as one
// group of asynchronous copies that overlaps the work issued after it: the data is in place after every
// thread's fz_cp_wait and a barrier, and X must not be read or written by the CTA until then.
__device__ void fz_stage_async(const float* __restrict__ G, int nb, int r0, int N, float* X, int ldx) {
  const int per_row = nb * (FZ / 2);  // float2 slots per row
  for (int e = threadIdx.x; e < FZ * per_row; e += blockDim.x) {
    const int i = e / per_row, q = e - i * per_row, blk = q / (FZ / 2), k = 2 * (q - blk * (FZ / 2));
    const bool real = i < N && k < N;
    fz_cp8(&X[i * ldx + blk * FZ + k], real ? G + (int64_t)(r0 + i) * nb * N + blk * N + k : G, real);
  }
  fz_cp_commit();
}

inline size_t fz_tl_smem() { return (size_t)(2 * FZ * FL1 + 2 * FZ * FL2 + 2 * FZ) * sizeof(float); }
inline size_t fz_relax_smem() { return (size_t)(2 * FZ * FL1 + 2 * FZ * FL2 + 2 * FZ) * sizeof(float); }

// T = S Ten and L = P T at operator slot s (k_dense.cuh's OpT32 and OpL32): T[i][j] = sum_h t_h(j) sum_k
// S[i][h N + k] D_s[k][j], L[i][j] = sum_h t_h(i) sum_k D_s[i][k] T[h N + k][j] (t_0 = x_s, t_1 = y_s), one row
// block h' of S and T (the x or the y rows) at a time. One CTA of FUSED_THREADS per vesicle (N <= 64); vesicles
// with active[v] == 0 are skipped when active is set.
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_fused_tl(OpCtx c, int s, const int* __restrict__ active) {
  extern __shared__ __align__(16) float fz[];
  float* Ds = fz;                        // [FZ][FL1]
  float* Tr = Ds + FZ * FL1;             // [FZ][FL1]: one row block of T
  float* Sr = Tr + FZ * FL1;             // [2][FZ][FL2]: the two row blocks of S, columns embedded
  float* txs = Sr + 2 * FZ * FL2;        // [FZ]
  float* tys = txs + FZ;                 // [FZ]
  const int v = c.vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = c.vi.N[v];
  const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
  const float* S = c.mat32(v, N, MatLayout::slot(s) + MatLayout::S);
  fz_stage_async(S, 2, 0, N, Sr, FL2);            // both row blocks of S in flight while D_s is formed
  fz_stage_async(S, 2, N, N, Sr + FZ * FL2, FL2);
  fz_load_ds(c, v, N, Ds, txs, tys);
  float* Tg = c.mat32(v, N, MatLayout::slot(s) + MatLayout::T);
  float lacc[8][2];
  fz_zero(lacc);
  for (int hp = 0; hp < 2; ++hp) {
    if (hp == 0) fz_cp_wait<1>(); else fz_cp_wait<0>();
    __syncthreads();  // S row block hp and D_s in place; the previous row block's L product has read Tr
    const float* X = Sr + hp * FZ * FL2;
    float tacc[8][2];
    fz_zero(tacc);
    for (int h = 0; h < 2; ++h) {
      float acc[8][2];
      fz_zero(acc);
      fz_gemm<2>(X + h * FZ, FL2, Ds, FL1, FZ, acc);
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float t = (h ? tys : txs)[2 * tc + b];
#pragma unroll
        for (int a = 0; a < 8; ++a) tacc[a][b] = fmaf(acc[a][b], t, tacc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = 8 * tr + a;
      *reinterpret_cast<float2*>(&Tr[i * FL1 + 2 * tc]) = make_float2(tacc[a][0], tacc[a][1]);
      if (i < N && 2 * tc < N)
        *reinterpret_cast<float2*>(Tg + (int64_t)(hp * N + i) * N + 2 * tc) = make_float2(tacc[a][0], tacc[a][1]);
    }
    __syncthreads();
    float acc[8][2];
    fz_zero(acc);
    fz_gemm<2>(Ds, FL1, Tr, FL1, FZ, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const float t = (hp ? tys : txs)[8 * tr + a];
#pragma unroll
      for (int b = 0; b < 2; ++b) lacc[a][b] = fmaf(acc[a][b], t, lacc[a][b]);
    }
  }
  float* Lg = c.mat32(v, N, MatLayout::slot(s) + MatLayout::L);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = 8 * tr + a;
    if (i < N && 2 * tc < N) *reinterpret_cast<float2*>(Lg + (int64_t)i * N + 2 * tc) = make_float2(lacc[a][0], lacc[a][1]);
  }
}

// W = L^{-1} (P B) and A = I - dt (B - T W) with B = -kappa S blockdiag(D4, D4), D4 = (D_s D_s)(D_s D_s), from
// S, T and the FP32 inverse of L at slot s (k_dense.cuh's OpD2_32 .. OpA32). B is formed one row block at a time
// (written to the B block, where the last stage reads it back), P B accumulates over the row blocks; W goes to the
// W block and A to the A block (inverted in place afterwards). One CTA of FUSED_THREADS per vesicle (N <= 64).
__global__ void __launch_bounds__(FUSED_THREADS, 2) k_fused_relax(OpCtx c, int s, float kappa, float dt,
                                                                  const int* __restrict__ active) {
  extern __shared__ __align__(16) float fz[];
  float* Ds = fz;                    // [FZ][FL1]: D_s, then a row block of T
  float* R = Ds + FZ * FL1;          // [FZ][FL1]: D2, then D4, then L^{-1}
  float* X = R + FZ * FL1;           // [FZ][FL2]: a row block of S, then P B
  float* Y = X + FZ * FL2;           // [FZ][FL2]: a row block of B, then W
  float* txs = Y + FZ * FL2;
  float* tys = txs + FZ;
  const int v = c.vi.vid(blockIdx.x);
  if (active && !active[v]) return;
  const int N = c.vi.N[v];
  const int tr = threadIdx.x >> 5, tc = threadIdx.x & 31;
  const float* S = c.mat32(v, N, MatLayout::slot(s) + MatLayout::S);
  const float* Tg = c.mat32(v, N, MatLayout::slot(s) + MatLayout::T);
  float* Bg = c.mat32(v, N, MatLayout::B);
  fz_stage_async(S, 2, 0, N, X, FL2);  // S row block 0 in flight while D4 is formed
  fz_load_ds(c, v, N, Ds, txs, tys);
  __syncthreads();
  {  // D2 = D_s D_s, then D4 = D2 D2 in place
    float acc[8][2];
    fz_zero(acc);
    fz_gemm<2>(Ds, FL1, Ds, FL1, FZ, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a) *reinterpret_cast<float2*>(&R[(8 * tr + a) * FL1 + 2 * tc]) = make_float2(acc[a][0], acc[a][1]);
    __syncthreads();
    fz_zero(acc);
    fz_gemm<2>(R, FL1, R, FL1, FZ, acc);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 8; ++a) *reinterpret_cast<float2*>(&R[(8 * tr + a) * FL1 + 2 * tc]) = make_float2(acc[a][0], acc[a][1]);
  }
  float pacc[8][4];
  fz_zero(pacc);
  for (int hp = 0; hp < 2; ++hp) {
    fz_cp_wait<0>();
    __syncthreads();  // S row block hp and D4 in place; the previous row block's P B product has read Y
    for (int h = 0; h < 2; ++h) {  // row block hp of B = -kappa S blockdiag(D4, D4)
      float acc[8][2];
      fz_zero(acc);
      fz_gemm<2>(X + h * FZ, FL2, R, FL1, FZ, acc);
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int i = 8 * tr + a;
        const float2 bv = make_float2(-kappa * acc[a][0], -kappa * acc[a][1]);
        *reinterpret_cast<float2*>(&Y[i * FL2 + h * FZ + 2 * tc]) = bv;
        if (i < N && 2 * tc < N) *reinterpret_cast<float2*>(Bg + (int64_t)(hp * N + i) * 2 * N + h * N + 2 * tc) = bv;
      }
    }
    __syncthreads();  // X and R have been read
    if (hp == 0)
      fz_stage_async(S, 2, N, N, X, FL2);                                           // S row block 1
    else
      fz_stage_async(c.mat32(v, N, MatLayout::slot(s) + MatLayout::L), 1, 0, N, R, FL1);  // L^{-1}
    float acc[8][4];  // P B += diag(t_hp) D_s B[row block hp], while the copy runs
    fz_zero(acc);
    fz_gemm<4>(Ds, FL1, Y, FL2, FZ, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const float t = (hp ? tys : txs)[8 * tr + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) pacc[a][b] = fmaf(acc[a][b], t, pacc[a][b]);
    }
  }
  __syncthreads();  // D_s has been read by the last P B product
  fz_stage_async(Tg, 1, 0, N, Ds, FL1);  // T row block 0, while W is formed
#pragma unroll
  for (int a = 0; a < 8; ++a)
    *reinterpret_cast<float4*>(&X[(8 * tr + a) * FL2 + 4 * tc]) = make_float4(pacc[a][0], pacc[a][1], pacc[a][2], pacc[a][3]);
  fz_cp_wait<1>();  // L^{-1} (the older group) has arrived
  __syncthreads();
  {  // W = L^{-1} (P B) into Y and the W block (N x 2N)
    float acc[8][4];
    fz_zero(acc);
    fz_gemm<4>(R, FL1, X, FL2, FZ, acc);
    float* Wg = c.mat32(v, N, MatLayout::W);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = 8 * tr + a;
      *reinterpret_cast<float4*>(&Y[i * FL2 + 4 * tc]) = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = fz_real(4 * tc + b, N);
        if (i < N && j >= 0) Wg[(int64_t)i * 2 * N + j] = acc[a][b];
      }
    }
  }
  float* Ag = c.mat32(v, N, MatLayout::A);
  for (int hp = 0; hp < 2; ++hp) {  // row block hp of A = I - dt (B - T W)
    if (hp == 1) {
      __syncthreads();  // the row block 0 product has read Ds
      fz_stage_async(Tg + (int64_t)N * N, 1, 0, N, Ds, FL1);
    }
    fz_cp_wait<0>();
    __syncthreads();
    float acc[8][4];
    fz_zero(acc);
    fz_gemm<4>(Ds, FL1, Y, FL2, FZ, acc);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = 8 * tr + a;
      if (i >= N) continue;
      const int64_t row = (int64_t)(hp * N + i) * 2 * N;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = fz_real(4 * tc + b, N);
        if (j < 0) continue;
        Ag[row + j] = ((hp * N + i == j) ? 1.f : 0.f) - dt * (Bg[row + j] - acc[a][b]);
      }
    }
  }
}

}  // namespace vs
