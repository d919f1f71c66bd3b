// Device helpers shared by the CUDA translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tnvan {

// Instance of block `blk` in a multi-instance launch (tiles of instance k are
// tile_begin[k] .. tile_begin[k+1]-1).
__device__ __forceinline__ int find_inst(const LaunchInfo& li, int blk) {
  int k = 0;
  while (k + 1 < li.n_inst && li.tile_begin[k + 1] <= blk) ++k;
  return k;
}

// Samples B of the batch that Eq. 10's weights -(l_b - mean l) / (beta B)
// divide by, from an instance's statistics row (written by the reduction or
// by tnvan_merge_stats): the finite l_b ([7]) plus the non-finite ones ([5]).
__device__ __forceinline__ double stats_batch(const double* st) { return st[7] + st[5]; }

// Philox step of a launch: the host value plus the optional device counter
// (lets a captured CUDA graph draw new numbers on every replay).
__device__ __forceinline__ uint32_t launch_step(const LaunchInfo& li) {
  return (uint32_t)(li.step + (li.step_dev ? *li.step_dev : 0ull));
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 round function
// with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += W0;
      k.y += W1;
    }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Power-of-two split m = f * 2^e with f in [1, 2) for a positive normal float;
// returns e.  Multiplying by pow2(-e) is exact.
__device__ __forceinline__ int exponent_of(float m) {
  return ((__float_as_int(m) >> 23) & 0xff) - 127;
}
__device__ __forceinline__ float pow2i(int e) {  // e in [-126, 127]
  return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ float softplusf(float z) {
  return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
}

// --- shared-memory barriers and bulk (TMA 1-D) copies --------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bounded wait for the phase with the given parity; false after max_iter polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int max_iter = 1 << 22) {
  for (int it = 0; it < max_iter; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Merge of two weighted branches in the moment form used for the
// magnetisation moments: each branch carries its (unnormalised) weight v, the
// conditional mean m and the conditional variance q of a sum over the
// branch's states.  The merged branch has weight v0 + v1, mean
// m1 + p0 (m0 - m1) and, by the law of total variance,
// q = p0 q0 + p1 q1 + p0 p1 (m0 - m1)^2 with p_i = v_i / (v0 + v1) -- the
// variance is never formed as a difference of raw second moments.  Zero
// total weight keeps branch 0 (any finite value: it is weighted by 0).
__device__ __forceinline__ void moment_mix(float v0, float m0, float q0, float v1, float m1, float q1, float& v,
                                           float& m, float& q) {
  const float vs = v0 + v1;
  if (vs > 0.f) {
    const float p0 = v0 / vs, p1 = v1 / vs, d = m0 - m1;
    m = fmaf(p0, d, m1);
    q = fmaf(p0, q0, p1 * q1) + p0 * p1 * d * d;
  } else {
    m = m0;
    q = q0;
  }
  v = vs;
}

}  // namespace tnvan
