// FP32 batched per-vesicle operator products on the tensor cores (tcgen05.mma, kind::f16, BF16 operands,
// FP32 accumulation in tensor memory). Each FP32 operand entry is split into three BF16 parts by
// successive rounding, x = x1 + x2 + x3 (24 significant bits together), and
//   C = x1 y1 + (x1 y2 + x2 y1) + (x1 y3 + x2 y2 + x3 y1)
// is accumulated in FP32; the dropped part products are below 2^-24 |x||y|, so C agrees with an FP32
// product to FP32 rounding. These products only build the preconditioners of the refinement (see the
// mixed-precision kernels), which need FP32 quality. At the per-vesicle sizes (m, n, K <= 2N) staging
// the functor-built operands in three parts costs more than the FP32 FMAs of k_bgemm save (measured:
// 1.7 ms for all products of a 2000 x 64 step with k_bgemm, 2.6 ms with this kernel), so it is opt-in.
//
// One CTA of 256 threads per (vesicle, 128 x 128 output tile); in the epilogue warp w reads the tensor-
// memory lanes 32 (w mod 4) onwards, warps 0-3 the columns 0-63 and warps 4-7 the columns 64-127. The
// operands come from the same functors as k_bgemm (so diagonal scalings and circulant entries are formed
// on the fly) and are staged in K
// chunks of 64 in the canonical no-swizzle K-major layout used by k_gemm_bf16 (core (g, c) of row group
// g and K-chunk c at byte (8 g + c) * 128). One elected thread issues the MMAs and commits them to an
// mbarrier; every wait has an iteration bound after which the kernel records ERR_MMA_TIMEOUT, skips the
// epilogue and still frees its tensor memory.
#pragma once
#include <cuda_bf16.h>

#include "k_dense.cuh"
#include "k_mlp.cuh"

namespace vs {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 64, TC_THREADS = 256;
constexpr int TC_PART = TC_BM * TC_BK * 2;   // bytes of one BF16 part of a 128 x 64 tile (16 KB)
constexpr int TC_SMEM = 6 * TC_PART + 1024;  // three parts of A and of B, plus alignment slack

__device__ __forceinline__ void split3(float x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// Stage rows [0, 128) x k in [kbase, kbase + 64) of a K-major operand, value(row, k) (0 outside), as
// three BF16 parts at dst, dst + TC_PART, dst + 2 TC_PART.
template <class F>
__device__ __forceinline__ void tc_stage(unsigned char* dst, int kbase, F value) {
  for (int e = threadIdx.x; e < TC_BM * 8; e += TC_THREADS) {
    const int r = e >> 3, cg = e & 7;
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) split3(value(r, kbase + 8 * cg + q), p0[q], p1[q], p2[q]);
    const int off = ((r >> 3) * 8 + cg) * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(p0);
    *reinterpret_cast<uint4*>(dst + TC_PART + off) = *reinterpret_cast<const uint4*>(p1);
    *reinterpret_cast<uint4*>(dst + 2 * TC_PART + off) = *reinterpret_cast<const uint4*>(p2);
  }
}

template <class Op>
__global__ void __launch_bounds__(TC_THREADS) k_bgemm_tc(Op op, const int* __restrict__ active, unsigned* err) {
  extern __shared__ unsigned char tc_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int v = op.c.vi.vid(blockIdx.z);
  if (active && !active[v]) return;
  const int N = op.c.vi.N[v];
  int m, n, K;
  op.dims(N, m, n, K);
  const int r0 = blockIdx.y * TC_BM, c0 = blockIdx.x * TC_BN;
  if (r0 >= m || c0 >= n) return;
  unsigned char* st = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = st;
  unsigned char* sb = st + 3 * TC_PART;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const int nk = (K + TC_BK - 1) / TC_BK;
  bool ok = true;
  for (int kb = 0; kb < nk; ++kb) {
    if (kb > 0) {  // the previous chunk's MMAs have read the staging buffers
      const bool w = mbar_wait(smem_addr(&mbar), (uint32_t)((kb - 1) & 1));
      if (__syncthreads_or(!w)) { ok = false; break; }
    }
    const int kbase = kb * TC_BK;
    tc_stage(sa, kbase, [&](int r, int k) {
      const int i = r0 + r;
      return (i < m && k < K) ? op.a(v, N, i, k) : 0.f;
    });
    tc_stage(sb, kbase, [&](int r, int k) {
      const int j = c0 + r;
      return (j < n && k < K) ? op.b(v, N, k, j) : 0.f;
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      // part pairs (A part, B part): the six products whose order is at most 2
      const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk)
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const uint64_t ad = umma_desc(smem_addr(sa + pa[t] * TC_PART) + kk * 256);
          const uint64_t bd = umma_desc(smem_addr(sb + pb[t] * TC_PART) + kk * 256);
          const uint32_t acc = (kb > 0 || kk > 0 || t > 0) ? 1u : 0u;
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                       ::"r"(tmem), "l"(ad), "l"(bd), "r"(MM_IDESC), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(&mbar)));
    }
  }
  if (ok && nk > 0) {
    const bool w = mbar_wait(smem_addr(&mbar), (uint32_t)((nk - 1) & 1));
    if (__syncthreads_or(!w)) ok = false;
  }
  if (!ok && tid == 0) atomicOr(err, ERR_MMA_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int wq = warp & 3, half = warp >> 2;
    const int i = r0 + wq * 32 + lane;
    for (int cc = half * (TC_BN / 2); cc < (half + 1) * (TC_BN / 2); cc += 16) {
      if (c0 + cc >= n) break;  // uniform across the warp
      uint32_t q[16];
      const uint32_t ta = tmem + ((uint32_t)(wq * 32) << 16) + (uint32_t)cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]), "=r"(q[7]),
            "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]), "=r"(q[14]), "=r"(q[15])
          : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (i < m) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c0 + cc + j;
          if (col < n) op.store(v, N, i, col, __uint_as_float(q[j]));
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
}

}  // namespace vs
