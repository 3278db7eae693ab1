// Counter-based random draws of the synthetic training-state generators
// (asse_learn.cu, asse_candidates.cu): SplitMix64 (Steele, Lea and Flood,
// 2014) keyed by a state's key and a draw index, and the murmur3 32-bit
// finaliser to make distinct bips.  A state is a pure function of (seed,
// index), so the tests can draw the same numbers on the host.
#pragma once

#include <cstdint>

namespace asse {

__device__ __forceinline__ uint64_t splitmix(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Draw i of the stream keyed by key: a double in [0, 1) from the top 53 bits.
__device__ __forceinline__ double unit(uint64_t key, uint64_t i)
{
    return (double)(splitmix(key ^ splitmix(i)) >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

}  // namespace asse
