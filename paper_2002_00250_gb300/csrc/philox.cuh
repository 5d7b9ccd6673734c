// philox.cuh -- Philox4x32-10 counter-based generator on the device.
//
// From the published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11): ten rounds; each round multiplies
// counter words 0 and 2 by the two Philox multipliers (32x32 -> 64 bit) and
// mixes the high halves with the other words and the key; the key is bumped by
// the two Weyl constants between rounds.
#pragma once
#include <cstdint>

namespace fos {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;  // multipliers
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;  // Weyl key bumps

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += kPhiloxW0;
            k.y += kPhiloxW1;
        }
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// The ten round keys of key k: rk[2r], rk[2r+1] = k + r * (W0, W1).
__host__ __device__ inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[20])
{
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + uint32_t(r) * kPhiloxW0;
        rk[2 * r + 1] = k1 + uint32_t(r) * kPhiloxW1;
    }
}

// The same generator with the round keys precomputed (the same bits as
// philox4x32_10(c, k) for rk from philox_round_keys(k)): when rk is a kernel
// parameter, every round mixes in its key straight from the constant bank.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t (&rk)[20])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ rk[2 * r], lo1, hi0 ^ c.w ^ rk[2 * r + 1], lo0);
    }
    return c;
}

}  // namespace fos
