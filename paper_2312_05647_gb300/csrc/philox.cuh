// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror &
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the
// uniform / normal draws the sampler and the surrogate take from it.
#pragma once

#include <cstdint>

namespace mjp {

// Ten rounds; each multiplies words 0 and 2 by the round multipliers, keeps
// both halves of the products and mixes the high halves with words 1, 3 and
// the key, which then advances by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// (m + 0.5) 2^-52 for the 52-bit m made of the top 26 bits of a and of b:
// exact in FP64 and strictly inside (0, 1).
__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) {
  return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-52;
}

// Box-Muller: two standard normals from two uniforms.
__device__ __forceinline__ void box_muller(double u1, double u2, double& z0, double& z1) {
  const double r = sqrt(-2.0 * log(u1));
  const double a = 2.0 * 3.141592653589793 * u2;
  z0 = r * cos(a);
  z1 = r * sin(a);
}

}  // namespace mjp
