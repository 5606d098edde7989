// shuffle.cuh -- the seeded per-epoch permutation of training samples used by
// the closure's minibatch gathers (closure_train.cu, mlp_train.cu).
#pragma once

#include <algorithm>

#include "internal.cuh"

namespace fp {

// Seeded permutation of [0, n) for one epoch: a four-round balanced Feistel
// network on 2*half bits (round function Philox4x32-7 keyed by the seed and
// counted by (right half, round, epoch)), which is a bijection of
// [0, 2^(2 half)), restricted to [0, n) by cycle walking (apply it again
// while the value is >= n).  The walk from a start below n ends at the first
// element of its cycle below n, after at most 2^(2 half) - n + 1 applications.
struct Perm {
    uint64_t n, limit;
    int half;
    uint32_t mask;
    uint2 key;
    uint32_t ep_lo, ep_hi;
};

__device__ __forceinline__ uint64_t feistel(uint64_t x, const Perm &p)
{
    uint32_t L = (uint32_t)(x >> p.half), R = (uint32_t)(x & p.mask);
#pragma unroll
    for (uint32_t round = 0; round < 4; ++round) {
        const uint4 h = philox4x32_7(make_uint4(R, round, p.ep_lo, p.ep_hi), p.key);
        const uint32_t nl = R;
        R = (L ^ h.x) & p.mask;
        L = nl;
    }
    return ((uint64_t)L << p.half) | R;
}

__device__ __forceinline__ uint64_t perm_index(uint64_t i, const Perm &p)
{
    uint64_t x = i;
    for (uint64_t it = 0; it < p.limit; ++it) {
        x = feistel(x, p);
        if (x < p.n) break;
    }
    return x;
}

inline Perm make_perm(int64_t n, uint64_t seed, int64_t epoch)
{
    Perm p{};
    p.n = (uint64_t)n;
    int bits = 0;
    while (bits < 62 && (1ull << bits) < (uint64_t)n) ++bits;
    bits = std::max(bits, 2);
    bits += bits & 1;
    p.half = bits / 2;
    p.mask = (uint32_t)((1ull << p.half) - 1);
    p.limit = (1ull << bits) - (uint64_t)n + 1;
    p.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    p.ep_lo = (uint32_t)epoch;
    p.ep_hi = (uint32_t)((uint64_t)epoch >> 32);
    return p;
}

}  // namespace fp
