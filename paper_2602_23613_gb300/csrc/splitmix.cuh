// Counter-based SplitMix64 draws (Steele, Lea, Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014): draw i of (stream, seed) is the first output of a SplitMix64 generator
// whose state is stream << 60 | seed << 40 | i; a U(0,1) double takes its top 53 bits.
#pragma once
#include <cstdint>

namespace amgh {

__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline double splitmix_u01(uint64_t stream, uint64_t seed, uint64_t i) {
    const uint64_t key = (stream << 60) | ((seed & 0xFFFFFull) << 40);
    return (double)(splitmix64(key + i) >> 11) * (1.0 / 9007199254740992.0);
}

constexpr uint64_t STREAM_MLP = 7, STREAM_PROBE = 8;

}  // namespace amgh
