// Counter-based sampling on the device.
//
// The paper's hash-based RNG (Sec. 3.1, Eq. hash_prob) combines one seed per
// random process with a hash of the process's current state; for walks the
// state is the current vertex and the walk length (Sec. 3.3, Eq. select-xor),
// and the walk id completes the key (Sec. 2.2).  Here:
//   walk key   K(seed, stream, k) = one half of Philox-4x32-10 applied to the
//              counter (k/2, stream) with key seed (Salmon et al., SC'11);
//              the even walk takes words 0-1, the odd walk words 2-3, so one
//              Philox block serves two consecutive walks;
//   step word  H = high 32 bits of SplitMix64's mixing function (Steele, Lea
//              and Flood, OOPSLA'14) applied to (K + l * golden) xor cur,
//              i.e. the l-th SplitMix64 state of seed K with the vertex folded
//              in;
//   choice     Eq. select-proposed with h_max = 2^32: k = (H * d) >> 32.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace bq {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMixA = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMixB = 0x94D049BB133111EBull;

struct Philox4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ Philox4 philox10(uint32_t c0, uint32_t c1, uint32_t c2,
                                            uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(kPhiloxM0, c0);
        const uint32_t lo0 = kPhiloxM0 * c0;
        const uint32_t hi1 = __umulhi(kPhiloxM1, c2);
        const uint32_t lo1 = kPhiloxM1 * c2;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return Philox4{c0, c1, c2, c3};
}

// Keys of walks 2j and 2j + 1 of `stream`.
__device__ __forceinline__ void walk_key_pair(uint64_t seed, uint64_t stream, uint64_t j,
                                              uint64_t &even, uint64_t &odd) {
    const Philox4 o = philox10((uint32_t)j, (uint32_t)(j >> 32), (uint32_t)stream,
                               (uint32_t)(stream >> 32), (uint32_t)seed,
                               (uint32_t)(seed >> 32));
    even = ((uint64_t)o.y << 32) | o.x;
    odd = ((uint64_t)o.w << 32) | o.z;
}

__device__ __forceinline__ uint64_t walk_key(uint64_t seed, uint64_t stream, uint64_t k) {
    uint64_t e, o;
    walk_key_pair(seed, stream, k >> 1, e, o);
    return (k & 1) ? o : e;
}

// `state` must be K + l * kGolden for step l.
__device__ __forceinline__ uint32_t step_word(uint64_t state, uint32_t cur) {
    uint64_t z = state ^ (uint64_t)cur;
    z = (z ^ (z >> 30)) * kMixA;
    z = (z ^ (z >> 27)) * kMixB;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}

__device__ __forceinline__ uint32_t choose(uint32_t r, uint32_t d) { return __umulhi(r, d); }

// Random word of the sampler: independent, or shared-top-bits coupling; or,
// with t == kSabaT, Eq. select-proposed literally: the walk's fixed seed xw
// xor the shared hash of (cur, l) (group_state is then one key for the batch).
template <bool COUPLED>
__device__ __forceinline__ uint32_t sample_word(uint64_t own_state, uint64_t group_state,
                                                uint32_t cur, uint32_t t, uint32_t xw = 0u) {
    if (!COUPLED) return step_word(own_state, cur);
    const uint32_t shared = step_word(group_state, cur);
    if (t == kSabaT) return shared ^ xw;
    return shared ^ (t >= 32 ? 0u : (step_word(own_state, cur) >> t));
}

}  // namespace bq
