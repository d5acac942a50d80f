// grpic_philox.cuh -- counter-based random numbers shared by the pair
// production of the batched lines and of the 2D grid: Philox4x64-10
// (Salmon, Moraes, Dror & Shaw, SC'11), a 53-bit uniform from its first
// word, and the splitmix64 finaliser (Steele, Lea & Flood 2014) for child ids.
#pragma once

#include <cstdint>

namespace grpic {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// the top 53 bits of the first output word for counter (id, step, event, 0)
// and key (seed, 0)
__device__ __forceinline__ uint64_t uniform53_bits(uint64_t seed, uint64_t id, int64_t step, int event)
{
    uint64_t c[4] = {id, (uint64_t)step, (uint64_t)event, 0ULL};
    philox4x64_10(c, seed, 0ULL);
    return c[0] >> 11;
}

// uniform in [0, 1): those bits times 2^-53
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t id, int64_t step, int event)
{
    return (double)uniform53_bits(seed, id, step, event) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t child_id(uint64_t parent, int64_t step, int k)
{
    return splitmix64(splitmix64(parent) ^ (((uint64_t)step << 2) | (uint64_t)k));
}

}  // namespace grpic
