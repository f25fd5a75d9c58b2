// rng.cuh -- SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) as a counter-based generator: output i of the stream started at
// `seed` is mix(seed + (i+1) * gamma), so any output can be computed on its own.
#pragma once
#include <stdint.h>

namespace hm {

__host__ __device__ __forceinline__ uint64_t splitmix64_out(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace hm
