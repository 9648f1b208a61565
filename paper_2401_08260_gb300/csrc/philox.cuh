// Counter-based random numbers of the library's draws (directions, random Fourier
// features).
#pragma once

#include <cstdint>

namespace slk {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy
// as 1, 2, 3", SC 2011): ten rounds of two 32x32->64 multiplies with the
// published round multipliers and Weyl key increments.
__device__ inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
        uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

// uniform in (0, 1) from 64 random bits (53-bit significand)
__device__ inline double u01(uint32_t hi, uint32_t lo) {
    unsigned long long v = (static_cast<unsigned long long>(hi) << 32) | lo;
    return (static_cast<double>(v >> 11) + 0.5) * 0x1.0p-53;
}

}  // namespace slk
