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

// Position of `key` in the sorted row[0, n), n >= 1: the largest i with
// row[i] <= key (0 if none), so the key is in the row iff row[i] == key.
// The trip count depends on n alone; the counting kernels search rows that
// every lane of a task shares (the task's start, or its edge's endpoints),
// so the loop never diverges.
__device__ __forceinline__ uint32_t last_le_row(const uint32_t *__restrict__ row, uint32_t n, uint32_t key) {
    uint32_t base = 0;
    while (n > 1) {
        const uint32_t half = n >> 1;
        if (__ldg(row + base + half) <= key) base += half;
        n -= half;
    }
    return base;
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
// counts (count + 1 entries, begin[count] = total tasks).  A direct-mapped
// bucket table indexed by task number replaces a binary search over the whole
// prefix (whose ~log2(count) dependent loads cost more than a short task's
// walks): with shift s = the least s such that (total >> s) <= count,
// bucket[b] = the edge holding task b << s, for the b with b << s < total (at
// most count + 1 entries).  Task t lies in an edge between bucket[t >> s] and
// bucket[(t >> s) + 1], a range that is about one edge on average, searched
// over contiguous entries of `begin`.
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

__host__ __device__ __forceinline__ uint32_t bucket_shift(uint64_t total, uint64_t count) {
    // least s with (total >> s) <= count: 2^s > total / (count + 1), i.e.
    // s = ceil(log2(q + 1)) for q = floor(total / (count + 1))
    const uint64_t q = total / (count + 1);
    uint32_t s = 0;
    while ((q >> s) != 0) ++s;
    return s;
}

__device__ __forceinline__ uint64_t task_edge(const uint64_t *__restrict__ begin, const uint32_t *__restrict__ bucket,
                                              uint64_t count, uint64_t total, uint32_t shift, uint64_t t) {
    const uint64_t b = t >> shift;
    const uint64_t lo = bucket[b];
    const uint64_t hi = ((b + 1) << shift) < total ? (uint64_t)bucket[b + 1] + 1 : count;
    return last_le_u64(begin, lo, hi, t);
}

// bucket[b] = e for every b with b << shift in [begin[e], begin[e + 1]).
// (A template so that each translation unit gets its own instance.)
template <int kUnused = 0>
__global__ void build_bucket_kernel(const uint64_t *__restrict__ begin, uint64_t count, uint32_t *__restrict__ bucket) {
    const uint64_t total = begin[count];
    const uint32_t shift = bucket_shift(total, count);
    const uint64_t step = 1ull << shift;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < count;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t lo = begin[e], hi = begin[e + 1];
        if (lo == hi) continue;
        for (uint64_t b = (lo + step - 1) >> shift; b <= ((hi - 1) >> shift); ++b) bucket[b] = (uint32_t)e;
    }
}

// Entries of the bucket table for `count` edges; edge indices are 32-bit.
inline uint64_t bucket_count(uint64_t count) { return count + 1; }
constexpr uint64_t kMaxBucketEdges = 0xffffffffull;

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
