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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace tnvan
