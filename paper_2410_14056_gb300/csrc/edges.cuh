// How a walk step reads the graph.  A step from a vertex with row offset
// `off` and degree `deg` picks index k < deg and needs, for the neighbour
// x = Gamma(cur)[k], the triple (x, row offset of x, degree of x) to take the
// next step.  Five layouts give that triple:
//   EdgesPackedIds  bit-packed id of x, then the 8-byte vertex record of x
//   EdgesCsr8       nbrs[j] then the 8-byte vertex record of x
//   EdgesCsr16      nbrs[j] then the 16-byte vertex record of x
//   EdgesPacked     one 8-byte edge record  {x | off << sh_off | deg << sh_deg}
//   EdgesWide       one 16-byte edge record {x, off lo, off hi, deg}
// The edge-record layouts make a step one dependent load instead of two but
// triple the bytes of the array read at random; on graphs that do not fit in
// L2 the packed ids (the smallest array) are fastest.
//
// Layouts with kSplit = true read the id and the vertex record separately
// (id(j), rec_of(x)), so a kernel may serve the record of a frequently
// visited vertex from shared memory instead.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace bq {

// L2 cache policies (createpolicy) and read-only loads that carry them.  The
// graph arrays a step reads at random are re-read all through a launch; the
// grouped walk ids and starts are read once.
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_normal() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t l2_policy_stream() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint4 ldg_pol(const uint4 *a, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(a), "l"(pol));
    return r;
}

__device__ __forceinline__ uint2 ldg_pol(const uint2 *a, uint64_t pol) {
    uint2 r;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(r.x), "=r"(r.y) : "l"(a), "l"(pol));
    return r;
}

__device__ __forceinline__ uint32_t ldg_pol(const uint32_t *a, uint64_t pol) {
    uint32_t r;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return r;
}

__device__ __forceinline__ void start_record(const int64_t *__restrict__ offsets, uint32_t v, uint64_t &off,
                                             uint32_t &deg) {
    const int64_t lo = __ldg(offsets + v);
    const int64_t hi = __ldg(offsets + v + 1);
    off = (uint64_t)lo;
    deg = (uint32_t)(hi - lo);
}

// Neighbour ids bit-packed q per 16-byte chunk (one aligned vector load), then
// the neighbour's 8-byte vertex record.  Shrinks the array a step reads at
// random so that more of it stays in L2.
struct EdgesPackedIds {
    static constexpr bool kSplit = true;
    const uint4 *pk;
    const uint2 *rec;
    uint32_t bits, q, mask;
    __device__ __forceinline__ uint32_t unpack(const uint4 &w, uint32_t bit) const {
        const uint32_t wi = bit >> 5, sh = bit & 31;
        const uint32_t lo = wi == 0 ? w.x : (wi == 1 ? w.y : (wi == 2 ? w.z : w.w));
        const uint32_t hi = wi == 0 ? w.y : (wi == 1 ? w.z : w.w);
        return __funnelshift_r(lo, hi, sh) & mask;
    }
    __device__ __forceinline__ uint32_t id(uint64_t j) const {
        const uint32_t jj = (uint32_t)j;  // built only when nnz < 2^32
        const uint32_t c = jj / q;
        return unpack(__ldg(pk + c), (jj - c * q) * bits);
    }
    __device__ __forceinline__ uint32_t id(uint64_t j, uint64_t pol) const {
        const uint32_t jj = (uint32_t)j;
        const uint32_t c = jj / q;
        return unpack(ldg_pol(pk + c, pol), (jj - c * q) * bits);
    }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint2 r = __ldg(rec + v);
        off = r.x;
        deg = r.y;
    }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg, uint64_t pol) const {
        const uint2 r = ldg_pol(rec + v, pol);
        off = r.x;
        deg = r.y;
    }
    __device__ __forceinline__ void next(uint64_t j, uint32_t &cur, uint64_t &off, uint32_t &deg) const {
        cur = id(j);
        rec_of(cur, off, deg);
    }
};

struct EdgesCsr8 {
    static constexpr bool kSplit = true;
    const uint32_t *nbrs;
    const uint2 *rec;
    __device__ __forceinline__ uint32_t id(uint64_t j) const { return __ldg(nbrs + j); }
    __device__ __forceinline__ uint32_t id(uint64_t j, uint64_t pol) const { return ldg_pol(nbrs + j, pol); }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint2 r = __ldg(rec + v);
        off = r.x;
        deg = r.y;
    }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg, uint64_t pol) const {
        const uint2 r = ldg_pol(rec + v, pol);
        off = r.x;
        deg = r.y;
    }
    __device__ __forceinline__ void next(uint64_t j, uint32_t &cur, uint64_t &off, uint32_t &deg) const {
        cur = id(j);
        rec_of(cur, off, deg);
    }
};

struct EdgesCsr16 {
    static constexpr bool kSplit = true;
    const uint32_t *nbrs;
    const uint4 *rec;
    __device__ __forceinline__ uint32_t id(uint64_t j) const { return __ldg(nbrs + j); }
    __device__ __forceinline__ uint32_t id(uint64_t j, uint64_t pol) const { return ldg_pol(nbrs + j, pol); }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint4 r = __ldg(rec + v);
        off = ((uint64_t)r.y << 32) | r.x;
        deg = r.z;
    }
    __device__ __forceinline__ void rec_of(uint32_t v, uint64_t &off, uint32_t &deg, uint64_t pol) const {
        const uint4 r = ldg_pol(rec + v, pol);
        off = ((uint64_t)r.y << 32) | r.x;
        deg = r.z;
    }
    __device__ __forceinline__ void next(uint64_t j, uint32_t &cur, uint64_t &off, uint32_t &deg) const {
        cur = id(j);
        rec_of(cur, off, deg);
    }
};

struct EdgesPacked {
    static constexpr bool kSplit = false;
    const uint64_t *e;
    uint32_t sh_off, sh_deg, mask_id;
    uint64_t mask_off;
    __device__ __forceinline__ void next(uint64_t j, uint32_t &cur, uint64_t &off, uint32_t &deg) const {
        const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(e) + j);
        cur = (uint32_t)w & mask_id;
        off = (w >> sh_off) & mask_off;
        deg = (uint32_t)(w >> sh_deg);
    }
};

struct EdgesWide {
    static constexpr bool kSplit = false;
    const uint4 *e;
    __device__ __forceinline__ void next(uint64_t j, uint32_t &cur, uint64_t &off, uint32_t &deg) const {
        const uint4 r = __ldg(e + j);
        cur = r.x;
        off = ((uint64_t)r.z << 32) | r.y;
        deg = r.w;
    }
};

// Task -> edge lookup.  `begin` is the exclusive prefix of per-edge task
// counts (count + 1 entries); `coarse[i] = begin[i * kTaskStride]`.  The
// search runs over the coarse array (small enough to stay in L2), then over
// at most kTaskStride contiguous entries of `begin`, instead of a binary search
// whose lower levels touch random lines of a large array.
constexpr uint32_t kTaskStride = 64;

__device__ __forceinline__ uint64_t last_le_u64(const uint64_t *__restrict__ a, uint64_t lo, uint64_t hi,
                                                uint64_t x) {
    // largest i in [lo, hi) with a[i] <= x, given a[lo] <= x
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint64_t task_edge(const uint64_t *__restrict__ begin, const uint64_t *__restrict__ coarse,
                                              uint64_t count, uint64_t t) {
    const uint64_t n_coarse = (count + kTaskStride - 1) / kTaskStride;
    const uint64_t c = last_le_u64(coarse, 0, n_coarse, t);
    const uint64_t lo = c * kTaskStride;
    const uint64_t hi = lo + kTaskStride < count ? lo + kTaskStride : count;
    return last_le_u64(begin, lo, hi, t);
}

// coarse[i] = begin[i * kTaskStride] for i < ceil(count / kTaskStride).
// (A template so that each translation unit gets its own instance.)
template <int kUnused = 0>
__global__ void build_coarse_kernel(const uint64_t *__restrict__ begin, uint64_t count, uint64_t *__restrict__ coarse) {
    const uint64_t n_coarse = (count + kTaskStride - 1) / kTaskStride;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_coarse;
         i += (uint64_t)gridDim.x * blockDim.x)
        coarse[i] = begin[i * kTaskStride];
}

inline uint64_t coarse_count(uint64_t count) { return (count + kTaskStride - 1) / kTaskStride; }

// Call f with the layout the graph was built with.
template <typename F>
int with_edges(const DeviceGraph &g, F &&f) {
    if (g.edge8) return f(EdgesPacked{g.edge8, g.sh_off, g.sh_deg, g.mask_id, g.mask_off});
    if (g.edge16) return f(EdgesWide{g.edge16});
    if (g.pk && g.rec8) return f(EdgesPackedIds{g.pk, g.rec8, g.pk_bits, g.pk_q, g.pk_mask});
    if (g.rec8) return f(EdgesCsr8{g.nbrs, g.rec8});
    return f(EdgesCsr16{g.nbrs, g.rec16});
}

}  // namespace bq
