// fp128.cuh -- device-side FP128 v1 primitives (the hash of Sec. 5.1's
// "hash of the data transferred", project-defined; the definition is in
// include/odp.h next to odp_fingerprint).
//
// Constants are produced at compile time from SplitMix64 (Steele, Lea,
// Flood 2014) seeded with 0x46503132385F7631; nothing is tabulated.
#pragma once

#include <stdint.h>

namespace odp {
namespace fp {

constexpr uint64_t kSeed = 0x46503132385F7631ull;

__host__ __device__ constexpr uint64_t splitmix(uint64_t seed, uint64_t i) {
    // the state after i + 1 golden-ratio increments, then the finaliser
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ constexpr uint64_t C(int i) { return splitmix(kSeed, (uint64_t)i); }
__host__ __device__ constexpr uint64_t Kodd(int i) { return C(i) | 1ull; }

// Compile-time names for the constants.
constexpr uint64_t KA1 = Kodd(0), KA2 = Kodd(1);   // chain a
constexpr uint64_t KB1 = Kodd(2), KB2 = Kodd(3);   // chain b
constexpr uint64_t KF1 = Kodd(4), KF2 = Kodd(5);   // lane finish
constexpr uint64_t KQ0 = Kodd(6), KQ1 = Kodd(7), KQ2 = Kodd(8), KQ3 = Kodd(9);
constexpr uint64_t KP0 = Kodd(10), KP1 = Kodd(11), KP2 = Kodd(12), KP3 = Kodd(13);
constexpr uint64_t KZ0 = Kodd(14), KZ1 = Kodd(15), KZ2 = Kodd(16), KZ3 = Kodd(17);
constexpr uint64_t D_LEAF_X = C(18), D_LEAF_Y = C(19);
constexpr uint64_t D_NODE = C(20), D_FINAL = C(21);
constexpr uint64_t EMPTY_X = C(22), EMPTY_Y = C(23);
constexpr int LANE_INIT_BASE = 32;  // lane l starts from C(32 + 2l), C(33 + 2l)

struct U128 {
    uint64_t x, y;
};

// Per-word chain step S(v; k1, k2).
__device__ __forceinline__ uint64_t chain(uint64_t v, uint64_t k1, uint64_t k2) {
    uint64_t t = v * k1;
    t ^= t >> 32;
    return t * k2;
}

template <uint64_t k0, uint64_t k1, uint64_t k2, uint64_t k3>
__device__ __forceinline__ U128 mix(uint64_t x, uint64_t y) {
    x *= k0;
    y ^= x >> 29;
    y *= k1;
    x ^= y >> 32;
    x *= k2;
    y ^= x >> 32;
    y *= k3;
    x ^= y >> 29;
    return U128{x, y};
}

// Leaf finalisation of a chunk root with r valid bytes.
__device__ __forceinline__ U128 leaf(uint64_t rx, uint64_t ry, uint64_t r) {
    return mix<KQ0, KQ1, KQ2, KQ3>(rx ^ r ^ D_LEAF_X, ry ^ D_LEAF_Y);
}

// Interior node of the leaf tree: left L, right R, `count` leaves below.
__device__ __forceinline__ U128 node(U128 L, U128 R, uint64_t count) {
    return mix<KP0, KP1, KP2, KP3>(L.x ^ R.y ^ count, L.y ^ R.x ^ R.y ^ D_NODE);
}

// Final output over the tree root.
__device__ __forceinline__ U128 finish(U128 root, uint64_t len, uint64_t nchunks) {
    return mix<KZ0, KZ1, KZ2, KZ3>(root.x ^ len, root.y ^ nchunks ^ D_FINAL);
}

__device__ __forceinline__ U128 empty_input() {
    return finish(U128{EMPTY_X, EMPTY_Y}, 0, 0);
}

// Lane start values, derived per lane at run time (no lane-indexed table).
__device__ __forceinline__ void lane_init(int lane, uint64_t& a, uint64_t& b) {
    a = splitmix(kSeed, (uint64_t)(LANE_INIT_BASE + 2 * lane));
    b = splitmix(kSeed, (uint64_t)(LANE_INIT_BASE + 2 * lane + 1));
}

}  // namespace fp
}  // namespace odp
