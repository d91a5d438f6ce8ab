// philox.cuh -- Philox4x32-10 counter-based generator for the device.
//
// Written from the generator's published definition (Salmon, Moraes, Dror,
// Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds,
// each multiplying counter words 0 and 2 by fixed odd constants (32x32 -> 64
// bits), mixing the high halves with words 1 and 3 and the key, and advancing
// the two key words by Weyl increments between rounds.
#pragma once
#include <cstdint>

namespace muca {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

}  // namespace muca

namespace muca {

// The same generator with the ten round keys of a fixed key computed once
// (k0 + i 0x9E3779B9, k1 + i 0xBB67AE85 for round i), for kernels that draw
// many blocks under one key.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__device__ __forceinline__ PhiloxKeys philox_keys(uint32_t k0, uint32_t k1)
{
    PhiloxKeys k;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        k.k0[round] = k0 + (uint32_t)round * 0x9E3779B9u;
        k.k1[round] = k1 + (uint32_t)round * 0xBB67AE85u;
    }
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.k0[round], lo1, hi0 ^ c.w ^ k.k1[round], lo0);
    }
    return c;
}

}  // namespace muca
