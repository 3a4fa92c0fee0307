// gg_hash.cuh - the hash that decides an arc's initial flag when the graph is
// sparsified (Sec. 3.4): SplitMix64 of the seed xor the arc's endpoints,
// compared with floor(sigma * 2^32).
#pragma once

#include <stdint.h>

namespace gg {

// SplitMix64 output for one state (Steele, Lea, Flood 2014): advance by the
// golden gamma, then the variant-13 finaliser.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long state)
{
    unsigned long long z = state + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial flag of arc src -> dst under ratio threshold thr = floor(sigma*2^32).
__device__ __forceinline__ uint32_t sampled_flag(int32_t src, int32_t dst, int symmetric,
                                                 unsigned long long seed, unsigned long long thr)
{
    uint32_t a = (uint32_t)src, b = (uint32_t)dst;
    if (symmetric && a > b) { uint32_t t = a; a = b; b = t; }
    const unsigned long long key = ((unsigned long long)a << 32) | b;
    return (splitmix64(seed ^ key) >> 32) < thr ? 1u : 0u;
}

}  // namespace gg
