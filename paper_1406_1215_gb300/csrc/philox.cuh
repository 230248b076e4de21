// philox.cuh -- Philox4x32-10 counter-based generator, written from its
// published description (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds; each round multiplies
// counter words 0 and 2 by the two round multipliers (high and low halves of
// the 64-bit products), xors the high halves with words 1 / 3 and the round
// key, and the two key words are bumped by the Weyl constants between rounds.
//
// The sampler's stream: key = (seed_lo, seed_hi), counter = (draw t,
// segment, u_lo, u_hi); one block per loop iteration of Algorithm 1.
#pragma once
#include <cstdint>

namespace cl {

struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  constexpr uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// The same with the round keys precomputed: rk[2r], rk[2r+1] = key + r * Weyl
// constants (round_keys below), so that a kernel parameter holds them.
__device__ __forceinline__ u32x4 philox4x32_10_rk(u32x4 c, const uint32_t (&rk)[20]) {
  constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = u32x4{hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0};
  }
  return c;
}

__host__ __device__ inline void round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[20]) {
  for (int r = 0; r < 10; ++r) {
    rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
    rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
  }
}

// The 52 random bits of a word pair: r = (2k+1) / 2^53 in (0, 1).
__device__ __forceinline__ unsigned long long grid52(uint32_t lo, uint32_t hi) {
  return (((unsigned long long)hi << 32) | lo) >> 12;
}

}  // namespace cl
