// rng.cuh -- counter-based random numbers of the library: SplitMix64
// (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014).  The generator adds gamma = 0x9E3779B97F4A7C15 to a 64-bit
// state and returns mix(state).  Stream (seed, ctr) starts at state
// s0 = seed XOR mix(ctr + gamma); its value number idx (0-based) is
// mix(s0 + (idx + 1) gamma), so any value can be drawn independently.
#pragma once
#include <stdint.h>

namespace mcl {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ULL;

__host__ __device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t cb_rand(uint64_t seed, uint64_t ctr, uint64_t idx) {
    const uint64_t s0 = seed ^ sm64_mix(ctr + kGamma);
    return sm64_mix(s0 + (idx + 1) * kGamma);
}

// uniform double in [0, 1) from the top 53 bits
__host__ __device__ __forceinline__ double cb_uniform(uint64_t seed, uint64_t ctr, uint64_t idx) {
    return (double)(cb_rand(seed, ctr, idx) >> 11) * 0x1.0p-53;
}

// standard normal number m: Box-Muller on values 2m (mapped into (0, 1]) and 2m+1
__device__ __forceinline__ double cb_normal(uint64_t seed, uint64_t ctr, uint64_t m) {
    const double u1 = ((double)(cb_rand(seed, ctr, 2 * m) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = cb_uniform(seed, ctr, 2 * m + 1);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

}  // namespace mcl
