// Learned part (Sec. 3.2, 3.4.2): BF16 tensor-core GEMMs with FP32 accumulation in tensor memory,
// fused epilogues, the paper's relative loss with its derivative term, and AdamW.
//
// k_gemm_bf16 computes D[m][n] = sum_k A[m][k] B[n][k] (both operands K-major, BF16) with
// tcgen05.mma (kind::f16, cta_group::1, M = 128, N = 128, K = 16 per instruction). One CTA per
// 128 x 128 output tile; its K loop stages 128 x 64 slices of A and B through a ring of MM_STAGES
// shared-memory buffers in the canonical no-swizzle K-major layout (8 x 8 core matrices, core (g, c)
// of row group g and K-chunk c at byte (8 g + c) * 128, so LBO = 128 B, SBO = 1024 B), filled by
// asynchronous 16-byte copies (cp.async) MM_STAGES - 1 slices ahead of the products; one elected thread
// issues the MMAs and commits them to the slice's mbarrier, which frees the buffer for its next fill, and
// the accumulator stays in 128 TMEM columns until the epilogue reads it back with tcgen05.ld. Every
// mbarrier wait has an iteration bound after which the kernel records an error, drains its copies and
// skips the epilogue.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace vs {

constexpr int MLP_MAX_OUT = 16384;  // widest layer


constexpr int MM_BM = 128, MM_BN = 128, MM_BK = 64, MM_THREADS = 128;
constexpr int MM_STAGE_BYTES = (MM_BM + MM_BN) * MM_BK * 2;   // 32 KB
constexpr int MM_STAGES = 4;                                 // shared-memory ring of K slices
constexpr int MM_SMEM = MM_STAGES * MM_STAGE_BYTES + 1024;   // the ring + 1 KB alignment slack
constexpr uint32_t MM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(MM_BN >> 3) << 17) |
                              ((uint32_t)(MM_BM >> 4) << 24);  // F32 accumulate, BF16 A and B, K-major
constexpr long long MM_WAIT_LIMIT = 1ll << 26;
enum : unsigned { ERR_MMA_TIMEOUT = 16u };

// epilogue: v = acc (+ bias[n]); RELU: max(v, 0); MASK: v * (mask[m][n] > 0); with oscale non-null
// v = v oscale[n] + oshift[n] (the network's output map); then write whichever of out_f32 [m][n],
// out_bf [m][n], out_bfT [n][m] is non-null.
enum : int { EPI_NONE = 0, EPI_RELU = 1, EPI_MASK = 2 };

struct GemmArgs {
  const __nv_bfloat16* A; int64_t lda;   // M x K
  const __nv_bfloat16* B; int64_t ldb;   // N x K
  int M, N, K;
  int act;
  const float* bias;                     // [N] or null
  float* out_f32; int64_t ld_f32;
  __nv_bfloat16* out_bf; int64_t ld_bf;
  __nv_bfloat16* out_bfT; int64_t ld_bfT;
  const __nv_bfloat16* mask; int64_t ld_mask;
  const float* oscale; const float* oshift;  // [N] each, or both null
  unsigned* err;
  // split K (kchunk > 0): CTA z of gridDim.z takes K range [z kchunk, (z + 1) kchunk) and writes its partial
  // product to out_f32 + z split_ld (no bias, activation or BF16 outputs)
  int kchunk; int64_t split_ld;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < MM_WAIT_LIMIT && !done; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  }
  return done != 0;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(__cvta_generic_to_global(src)),
               "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(MM_THREADS) k_gemm_bf16(GemmArgs g) {
  if (g.kchunk > 0) {
    const int k0 = blockIdx.z * g.kchunk;
    g.A += k0;
    g.B += k0;
    g.K = min(g.K - k0, g.kchunk);
    g.out_f32 += blockIdx.z * g.split_ld;
  }
  extern __shared__ unsigned char mm_raw[];
  __shared__ __align__(8) uint64_t mbar[MM_STAGES];
  __shared__ uint32_t tmem_base;
  unsigned char* st = (unsigned char*)(((uintptr_t)mm_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * MM_BM, n0 = blockIdx.x * MM_BN;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(MM_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < MM_STAGES; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[q])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nk = (g.K + MM_BK - 1) / MM_BK;
  // copies of K slice kb into ring buffer kb % MM_STAGES (out-of-range chunks are filled with zeros)
  auto fill = [&](int kb) {
    unsigned char* sa = st + (kb % MM_STAGES) * MM_STAGE_BYTES;
    unsigned char* sb = sa + MM_BM * MM_BK * 2;
    const int kbase = kb * MM_BK;
#pragma unroll
    for (int q = 0; q < MM_BM * 8 / MM_THREADS; ++q) {
      const int e = tid + q * MM_THREADS, r = e >> 3, c = e & 7;
      const int gm = m0 + r, gk = kbase + 8 * c;
      const bool in = gm < g.M && gk < g.K;
      cp_async16(smem_addr(sa + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16),
                 in ? (const void*)(g.A + (int64_t)gm * g.lda + gk) : (const void*)g.A, in ? 16u : 0u);
    }
#pragma unroll
    for (int q = 0; q < MM_BN * 8 / MM_THREADS; ++q) {
      const int e = tid + q * MM_THREADS, r = e >> 3, c = e & 7;
      const int gn = n0 + r, gk = kbase + 8 * c;
      const bool in = gn < g.N && gk < g.K;
      cp_async16(smem_addr(sb + ((r >> 3) * 8 + c) * 128 + (r & 7) * 16),
                 in ? (const void*)(g.B + (int64_t)gn * g.ldb + gk) : (const void*)g.B, in ? 16u : 0u);
    }
  };
#pragma unroll
  for (int p = 0; p < MM_STAGES - 1; ++p) {
    if (p < nk) fill(p);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  bool ok = true;
  for (int kb = 0; kb < nk; ++kb) {
    // slice kb has landed (this thread's copies, then everyone's), visible to the tensor core's proxy
    asm volatile("cp.async.wait_group %0;" ::"n"(MM_STAGES - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int s = kb % MM_STAGES;
    unsigned char* sa = st + s * MM_STAGE_BYTES;
    unsigned char* sb = sa + MM_BM * MM_BK * 2;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int kk = 0; kk < MM_BK / 16; ++kk) {
        const uint64_t ad = umma_desc(smem_addr(sa) + kk * 256);
        const uint64_t bd = umma_desc(smem_addr(sb) + kk * 256);
        const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(ad), "l"(bd), "r"(MM_IDESC), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar[s])));
    }
    // refill the buffer of slice kb - 1 with slice kb + MM_STAGES - 1 once its products are done
    const int nx = kb + MM_STAGES - 1;
    if (nx < nk) {
      if (kb >= 1) {
        const int pb = kb - 1;
        const bool w = mbar_wait(smem_addr(&mbar[pb % MM_STAGES]), (uint32_t)(pb / MM_STAGES) & 1u);
        if (__syncthreads_or(!w)) { ok = false; break; }
      }
      fill(nx);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");  // no copy left in flight, also after a timeout
  if (ok && nk > 0) {
    const int lb = nk - 1;
    const bool w = mbar_wait(smem_addr(&mbar[lb % MM_STAGES]), (uint32_t)(lb / MM_STAGES) & 1u);
    if (__syncthreads_or(!w)) ok = false;
  }
  if (!ok && tid == 0) atomicOr(g.err, ERR_MMA_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int r = warp * 32 + lane;
    const int gm = m0 + r;
    // whole 16-column chunks with 16-byte aligned rows (dims are multiples of 16) take the vector path
    const bool vec = (g.N % 16 == 0) && (!g.out_f32 || (g.ld_f32 % 4 == 0 && ((uintptr_t)g.out_f32 & 15) == 0)) &&
                     (!g.out_bf || (g.ld_bf % 8 == 0 && ((uintptr_t)g.out_bf & 15) == 0)) &&
                     (!g.bias || ((uintptr_t)g.bias & 15) == 0) &&
                     (g.act != EPI_MASK || (g.ld_mask % 8 == 0 && ((uintptr_t)g.mask & 15) == 0));
    for (int c0 = 0; c0 < MM_BN; c0 += 16) {
      if (n0 + c0 >= g.N) break;  // uniform across the CTA
      uint32_t v[16];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (gm < g.M) {
        const int gn0 = n0 + c0;
        float x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(v[j]);
        if (vec) {  // 16 whole, 16-element aligned columns: vector loads and stores of the row's chunk
          if (g.bias) {
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 b4 = *reinterpret_cast<const float4*>(g.bias + gn0 + j);
              x[j] += b4.x; x[j + 1] += b4.y; x[j + 2] += b4.z; x[j + 3] += b4.w;
            }
          }
          if (g.act == EPI_RELU) {
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = fmaxf(x[j], 0.f);
          }
          if (g.act == EPI_MASK) {
            __align__(16) __nv_bfloat16 mk[16];
            const uint4* msrc = reinterpret_cast<const uint4*>(g.mask + (int64_t)gm * g.ld_mask + gn0);
            *reinterpret_cast<uint4*>(mk) = msrc[0];
            *reinterpret_cast<uint4*>(mk + 8) = msrc[1];
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (!(__bfloat162float(mk[j]) > 0.f)) x[j] = 0.f;
          }
          if (g.oscale) {
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], g.oscale[gn0 + j], g.oshift[gn0 + j]);
          }
          if (g.out_f32) {
            float4* o = reinterpret_cast<float4*>(g.out_f32 + (int64_t)gm * g.ld_f32 + gn0);
#pragma unroll
            for (int j = 0; j < 4; ++j) o[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
          }
          __align__(16) __nv_bfloat16 bv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) bv[j] = __float2bfloat16_rn(x[j]);
          if (g.out_bf) {
            uint4* o = reinterpret_cast<uint4*>(g.out_bf + (int64_t)gm * g.ld_bf + gn0);
            o[0] = *reinterpret_cast<const uint4*>(bv);
            o[1] = *reinterpret_cast<const uint4*>(bv + 8);
          }
          if (g.out_bfT) {
#pragma unroll
            for (int j = 0; j < 16; ++j) g.out_bfT[(int64_t)(gn0 + j) * g.ld_bfT + gm] = bv[j];
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int gn = gn0 + j;
            if (gn >= g.N) break;
            float y = x[j];
            if (g.bias) y += g.bias[gn];
            if (g.act == EPI_RELU) y = fmaxf(y, 0.f);
            if (g.act == EPI_MASK && !(__bfloat162float(g.mask[(int64_t)gm * g.ld_mask + gn]) > 0.f)) y = 0.f;
            if (g.oscale) y = fmaf(y, g.oscale[gn], g.oshift[gn]);
            if (g.out_f32) g.out_f32[(int64_t)gm * g.ld_f32 + gn] = y;
            const __nv_bfloat16 b = __float2bfloat16_rn(y);
            if (g.out_bf) g.out_bf[(int64_t)gm * g.ld_bf + gn] = b;
            if (g.out_bfT) g.out_bfT[(int64_t)gn * g.ld_bfT + gm] = b;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MM_BN));
}

// FP32 rows (batch x d) -> BF16 rows and BF16 transposed (d x Bp), zero rows for batch <= b < Bp.
// With shift non-null each feature is first mapped to (x[j] - shift[j]) scale[j] in FP32 (the network's
// input map).
__global__ void k_rows_to_bf16(const float* __restrict__ x, int batch, int Bp, int d, const float* __restrict__ shift,
                               const float* __restrict__ scale, __nv_bfloat16* __restrict__ out,
                               __nv_bfloat16* __restrict__ outT) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)Bp * d) return;
  const int b = (int)(e / d), j = (int)(e - (int64_t)b * d);
  float xv = b < batch ? x[e] : 0.f;
  if (shift && b < batch) xv = __fmul_rn(__fsub_rn(xv, shift[j]), scale[j]);
  const __nv_bfloat16 v = __float2bfloat16_rn(xv);
  out[e] = v;
  outT[(int64_t)j * Bp + b] = v;
}

// Per-sample loss (Sec. 3.4.2) and its gradient: one CTA per sample row b.
//   loss_b = ||e|| / ||y|| + beta ||D e|| / ||D y||,  e = yhat - y,
// where, with yshift non-null, y is the target in the network's output coordinates,
// (target[j] - yshift[j]) yinv[j] in FP32, and yhat is the output before the output map.
//   D = periodic forward difference inside each of ncomp equal blocks of the row;
//   dL/dyhat = (e / (||e|| ||y||) + beta D^T D e / (||D e|| ||D y||)) / batch.
__global__ void __launch_bounds__(128) k_mlp_loss(const float* __restrict__ yhat, const float* __restrict__ yraw,
                                                  const float* __restrict__ yshift, const float* __restrict__ yinv,
                                                  float* __restrict__ y, int batch,
                                                  int d, int ncomp, float beta, float* __restrict__ g_f32,
                                                  __nv_bfloat16* __restrict__ g_bf, __nv_bfloat16* __restrict__ g_bfT,
                                                  int Bp, float* __restrict__ loss_b) {
  __shared__ double red[4];
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  const int n = d / ncomp;
  if (b >= batch) {
    for (int j = tid; j < d; j += blockDim.x) {
      g_f32[(int64_t)b * d + j] = 0.f;
      g_bf[(int64_t)b * d + j] = __float2bfloat16_rn(0.f);
      g_bfT[(int64_t)j * Bp + b] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  // y: the row's targets in output coordinates (a scratch row when yshift is set, else yraw itself)
  if (yshift) {
    for (int j = tid; j < d; j += blockDim.x)
      y[(int64_t)b * d + j] = __fmul_rn(__fsub_rn(yraw[(int64_t)b * d + j], yshift[j]), yinv[j]);
    __syncthreads();
  } else {
    y = const_cast<float*>(yraw);
  }
  // errors e_j and periodic differences de_j = e_{next(j)} - e_j within each component's block, recomputed
  // from global memory where needed (rows up to MLP_MAX_OUT wide)
  const float* yh = yhat + (int64_t)b * d;
  const float* yr = y + (int64_t)b * d;
  auto err = [&](int j) { return yh[j] - yr[j]; };
  auto nxt = [&](int j) { const int blk = j / n, k = j - blk * n; return blk * n + ((k + 1 == n) ? 0 : k + 1); };
  auto prv = [&](int j) { const int blk = j / n, k = j - blk * n; return blk * n + ((k == 0) ? n - 1 : k - 1); };
  double se = 0.0, sy = 0.0, sde = 0.0, sdy = 0.0;
  for (int j = tid; j < d; j += blockDim.x) {
    const float t = yr[j], e = err(j);
    se += (double)e * e;
    sy += (double)t * t;
    const int nx = nxt(j);
    const float de = err(nx) - e;
    const float dy = yr[nx] - t;
    sde += (double)de * de;
    sdy += (double)dy * dy;
  }
  se = block_sum(se, red);
  sy = block_sum(sy, red);
  sde = block_sum(sde, red);
  sdy = block_sum(sdy, red);
  const double ne = sqrt(se), ny = sqrt(sy), nde = sqrt(sde), ndy = sqrt(sdy);
  if (tid == 0) loss_b[b] = (float)(ne / ny + beta * nde / ndy);
  const double c1 = ne > 0 ? 1.0 / (ne * ny * batch) : 0.0;
  const double c2 = nde > 0 ? beta / (nde * ndy * batch) : 0.0;
  for (int j = tid; j < d; j += blockDim.x) {
    const int pv = prv(j);
    const float e = err(j), de = err(nxt(j)) - e, dep = e - err(pv);
    const float gv = (float)(c1 * e + c2 * ((double)dep - de));
    g_f32[(int64_t)b * d + j] = gv;
    const __nv_bfloat16 bv = __float2bfloat16_rn(gv);
    g_bf[(int64_t)b * d + j] = bv;
    g_bfT[(int64_t)j * Bp + b] = bv;
  }
}

// Column mean and standard deviation of a row-major FP32 matrix (rows x cols), FP64 sums in a fixed
// order, one thread per column: mean[c], and sd[c] = sqrt(mean of squared deviations).
__global__ void k_colstats(const float* __restrict__ X, int rows, int cols, double* __restrict__ mean,
                           double* __restrict__ sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += X[(int64_t)r * cols + c];
  const double m = s / rows;
  double q = 0.0;
  for (int r = 0; r < rows; ++r) {
    const double d = X[(int64_t)r * cols + c] - m;
    q += d * d;
  }
  mean[c] = m;
  sd[c] = sqrt(q / rows);
}

// Mean of the per-sample losses (fixed order, one thread).
__global__ void k_mean(const float* __restrict__ v, int n, float* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = (float)(s / n);
  }
}

// db[n] = sum_b G[b][n] (fixed order per column).
__global__ void k_colsum(const float* __restrict__ G, int rows, int cols, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += G[(int64_t)r * cols + c];
  out[c] = s;
}

// AdamW on the flat FP32 master parameters (decoupled weight decay).
__global__ void k_adamw(float* __restrict__ w, const float* __restrict__ gr, float* __restrict__ m, float* __restrict__ v,
                        int64_t n, float lr, float b1, float b2, float eps, float wd, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / c1, vh = vi / c2;
  w[i] = w[i] * (1.f - lr * wd) - lr * mh / (sqrtf(vh) + eps);
}

// BF16 copies W (rows x cols) and W^T (cols x rows) of an FP32 weight matrix.
__global__ void k_weights_bf16(const float* __restrict__ W, int rows, int cols, __nv_bfloat16* __restrict__ Wb,
                               __nv_bfloat16* __restrict__ WbT) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e - (int64_t)r * cols);
  const __nv_bfloat16 b = __float2bfloat16_rn(W[e]);
  Wb[e] = b;
  WbT[(int64_t)c * rows + r] = b;
}

}  // namespace vs
