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

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += kW0;
            k.y += kW1;
        }
        const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
        const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

}  // namespace fos
