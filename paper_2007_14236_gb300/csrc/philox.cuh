// philox.cuh -- counter-based Philox4x32-10 random numbers on the device.
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw ("Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds, each multiplying words 0
// and 2 by the two Philox constants and xoring the high product halves with
// words 1 and 3 and the round key; the key advances by the two Weyl
// constants between rounds.
//
// Stream layout used by the library: key = (seed low, seed high), counter =
// (index low, index high, purpose | attempt << 8, stream).  Every draw is a
// pure function of its counter, so results do not depend on thread mapping.
#pragma once
#include <stdint.h>

namespace ngb {

struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ __forceinline__ U4 draw4(uint64_t seed, uint64_t index, uint32_t purpose, uint32_t attempt,
                                             uint32_t stream) {
  return philox4x32_10(U4{(uint32_t)index, (uint32_t)(index >> 32), purpose | (attempt << 8), stream},
                       (uint32_t)seed, (uint32_t)(seed >> 32));
}

// uniform integer in [0, n): high word of x * n
__host__ __device__ __forceinline__ uint32_t scale_index(uint32_t x, uint32_t n) {
  return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

// uniform double in (0, 1] from 53 bits of two words
__host__ __device__ __forceinline__ double unit53(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((((uint64_t)hi) << 32) | (uint64_t)lo) >> 11;
  return (double)(m + 1ull) * 1.1102230246251565e-16;  // 2^-53
}

#ifdef __CUDACC__
// Box-Muller (cosine branch) in FP64 with uncontracted operations.
__device__ __forceinline__ double gauss(U4 r) {
  const double u1 = unit53(r.x, r.y);
  const double u2 = unit53(r.z, r.w);
  const double rad = sqrt(__dmul_rn(-2.0, log(u1)));
  return __dmul_rn(rad, cos(__dmul_rn(6.283185307179586, u2)));
}
#endif

}  // namespace ngb
