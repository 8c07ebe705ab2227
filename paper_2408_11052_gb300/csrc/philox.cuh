// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11), device implementation.
//
// Ten rounds; each multiplies counter words 0 and 2 by the two Philox4x64
// multipliers, takes the 128-bit products' high and low halves, mixes the
// high halves with counter words 1 and 3 and the round key, and permutes.
// The key advances by the two Weyl increments between rounds.
#pragma once

#include <stdint.h>

namespace crl {

struct Philox4 {
  unsigned long long w[4];
};

__device__ __forceinline__ Philox4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                                 unsigned long long c2, unsigned long long c3,
                                                 unsigned long long k0, unsigned long long k1) {
  constexpr unsigned long long M0 = 0xD2E7470EE14C6C93ull;
  constexpr unsigned long long M1 = 0xCA5A826395121157ull;
  constexpr unsigned long long W0 = 0x9E3779B97F4A7C15ull;
  constexpr unsigned long long W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    const unsigned long long n0 = hi1 ^ c1 ^ k0;
    const unsigned long long n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  Philox4 r;
  r.w[0] = c0;
  r.w[1] = c1;
  r.w[2] = c2;
  r.w[3] = c3;
  return r;
}

// Uniform double in (0, 1) from the top 53 bits of a word (never 0).
__device__ __forceinline__ double u64_to_unit_open(unsigned long long x) {
  return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

// N(0, 1) draw for element d of row b: Box-Muller on the block (step, b, word, d / 4);
// words (0, 1) feed elements 4q, 4q+1 and words (2, 3) feed 4q+2, 4q+3 (cos /
// sin branch).  `word` separates the streams (1: the actor's noise; the
// collection stub takes 2 to 5).  T = double draws in double, float in float
// (the same Philox words, so the two agree to float rounding).
template <typename T>
__device__ T philox_normal(unsigned long long step, int b, unsigned long long word, int d, unsigned long long seed,
                           unsigned long long agent) {
  constexpr double kTwoPi = 6.28318530717958647693;
  const Philox4 r = philox4x64_10(step, (unsigned long long)b, word, (unsigned long long)(d / 4), seed, agent);
  const bool pair = (d % 4) >= 2;   // words 0, 1 or 2, 3 (selected, not indexed: no local array)
  const double u1 = u64_to_unit_open(pair ? r.w[2] : r.w[0]);
  const double u2 = u64_to_unit_open(pair ? r.w[3] : r.w[1]);
  if constexpr (sizeof(T) == 8) {
    const double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincos(kTwoPi * u2, &s, &c);
    return (d % 2 == 0) ? rad * c : rad * s;
  } else {
    const float rad = sqrtf(-2.0f * logf((float)u1));
    float s, c;
    sincosf((float)(kTwoPi * u2), &s, &c);
    return (d % 2 == 0) ? rad * c : rad * s;
  }
}

}  // namespace crl
