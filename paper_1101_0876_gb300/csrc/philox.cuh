// Device-side Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11).
//
// Per round: the 64-bit products of counter word 0 and word 2 with two
// fixed multipliers are formed, and the new counter is
//   (hi(m1*c2) ^ c1 ^ k0, lo(m1*c2), hi(m0*c0) ^ c3 ^ k1, lo(m0*c0)).
// The key advances by two Weyl constants between rounds (nine bumps over
// ten rounds).  The key is the same for every thread of a launch, so the
// ten round keys are formed once (uniform values) and each round costs two
// wide multiplies and two three-input XORs per thread.
#pragma once
#include <cstdint>

namespace potts {

struct PhiloxKey {
  uint32_t k0[10];
  uint32_t k1[10];
};

__host__ __device__ __forceinline__ PhiloxKey philox_schedule(uint32_t key0,
                                                              uint32_t key1) {
  PhiloxKey s;
  for (int r = 0; r < 10; ++r) {
    s.k0[r] = key0 + (uint32_t)r * 0x9E3779B9u;
    s.k1[r] = key1 + (uint32_t)r * 0xBB67AE85u;
  }
  return s;
}

__device__ __forceinline__ uint4 philox10(uint32_t c0, uint32_t c1,
                                          uint32_t c2, uint32_t c3,
                                          const PhiloxKey &ks) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ ks.k0[r];
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ ks.k1[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return make_uint4(c0, c1, c2, c3);
}

}  // namespace potts
