// Walk-batch kernels: Alg. 2 (RandomWalk, one walk per thread: the naive
// plain form) and Alg. 3 (RandomBouquet: the walks of one start vertex
// advanced in lockstep by the lanes of a warp), with visit counting as in the
// synthetic benchmark of Sec. 4 and the hash-keyed choice of Eq.
// select-proposed.
//
// Both kernels compute exactly the same integer visit counts: walk i's path
// depends only on (seed, i, start, graph); only the order in which the walks
// are executed differs.
//
// Memory per step (the random gathers Sec. 3.2 names as the bottleneck): the
// naive kernel reads the 4-byte neighbour id and the neighbour's 8-byte
// vertex record (two dependent loads); the bouquet kernel, on graphs built
// with edge records, reads one 8-byte edge record.  Plus a 4-byte visit
// atomic.
#include <algorithm>

#include <cooperative_groups.h>

#include "edges.cuh"
#include "hash.cuh"
#include "internal.h"

namespace bq {
namespace cg = cooperative_groups;

namespace {

constexpr int kThreads = 256;

struct RecCompact {
    const uint2 *rec;
    __device__ __forceinline__ void load(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint2 r = __ldg(rec + v);
        off = r.x;
        deg = r.y;
    }
};

struct RecWide {
    const uint4 *rec;
    __device__ __forceinline__ void load(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint4 r = __ldg(rec + v);
        off = ((uint64_t)r.y << 32) | r.x;
        deg = r.z;
    }
};

__device__ __forceinline__ void add_visits(uint32_t *visits, uint32_t v, uint32_t inc, bool checked,
                                           uint32_t *status) {
    if (checked) {
        const uint32_t old = atomicAdd(visits + v, inc);
        if (old + inc < old) atomicOr(status, kStatusOverflow);
    } else {
        atomicAdd(visits + v, inc);
    }
}

// -------------------------------------------------------------- naive

template <typename RL, bool COUPLED>
__global__ void __launch_bounds__(kThreads)
walk_naive_kernel(RL rl, const uint32_t *__restrict__ nbrs, uint32_t n, const uint32_t *__restrict__ starts,
                  uint64_t n_walks, uint32_t n_steps, uint64_t seed, Sampler smp, bool visit_start,
                  bool checked, uint32_t *__restrict__ visits, uint32_t *__restrict__ paths,
                  uint32_t *status) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_walks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t cur = starts[i];
        if (cur >= n) {
            atomicOr(status, kStatusBadStart);
            continue;
        }
        uint64_t st = walk_key(seed, kBatchStream, i);
        const bool saba = COUPLED && smp.t == kSabaT;
        uint64_t gs = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, saba ? 0 : i / smp.width) : 0;
        const uint32_t xw = (uint32_t)st;
        uint32_t *row = paths ? paths + i * ((uint64_t)n_steps + 1) : nullptr;
        if (row) row[0] = cur;
        if (visit_start) add_visits(visits, cur, 1, checked, status);
        for (uint32_t l = 1; l <= n_steps; ++l) {
            st += kGolden;
            if (COUPLED) gs += kGolden;
            uint64_t off;
            uint32_t d;
            rl.load(cur, off, d);
            if (d) cur = nbrs[off + choose(sample_word<COUPLED>(st, gs, cur, smp.t, xw), d)];
            add_visits(visits, cur, 1, checked, status);
            if (row) row[l] = cur;
        }
    }
}

// ------------------------------------------------ grouping by start vertex

__global__ void hist_starts_kernel(const uint32_t *__restrict__ starts, uint64_t n_walks, uint32_t n,
                                   uint32_t *__restrict__ counts, uint32_t *status) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_walks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = starts[i];
        if (s < n) atomicAdd(counts + s, 1u);
        else atomicOr(status, kStatusBadStart);
    }
}

// cursor[v] starts at the first slot of v's bucket; walks of start v are
// placed in its bucket (order inside a bucket is unspecified and does not
// change any result).
__global__ void scatter_starts_kernel(const uint32_t *__restrict__ starts, uint64_t n_walks, uint32_t n,
                                      uint32_t *__restrict__ cursor, uint2 *__restrict__ sorted) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_walks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = starts[i];
        if (s >= n) continue;
        const uint32_t pos = atomicAdd(cursor + s, 1u);
        sorted[pos] = make_uint2((uint32_t)i, s);  // one 8-byte store
    }
}

// Without grouping (bq_tuning.group_walks = 0): the valid walks' (walk id,
// start) pairs in input order within each block's tile of kPairTile walks
// (one atomic per tile reserves its slots), their number in *n_valid;
// starts >= n are skipped and reported.  The order of the tiles follows the
// schedule; no result depends on it.
constexpr int kPairTile = 1024;  // = the block size

__global__ void __launch_bounds__(kPairTile)
pairs_in_order_kernel(const uint32_t *__restrict__ starts, uint64_t n_walks, uint32_t n,
                      uint32_t *__restrict__ n_valid, uint2 *__restrict__ sorted, uint32_t *status) {
    __shared__ uint32_t s_warp[kPairTile / 32];
    __shared__ uint32_t s_base;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint64_t tile = blockIdx.x * (uint64_t)kPairTile; tile < n_walks; tile += (uint64_t)gridDim.x * kPairTile) {
        const uint64_t i = tile + threadIdx.x;
        const uint32_t s = i < n_walks ? starts[i] : 0u;
        const bool valid = i < n_walks && s < n;
        if (i < n_walks && !valid) atomicOr(status, kStatusBadStart);
        const uint32_t mask = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) s_warp[warp] = (uint32_t)__popc(mask);
        __syncthreads();
        if (threadIdx.x == 0) {  // the tile's warps in order, then one atomic
            uint32_t acc = 0;
            for (int w = 0; w < kPairTile / 32; ++w) {
                const uint32_t c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_base = acc ? atomicAdd(n_valid, acc) : 0u;
        }
        __syncthreads();
        if (valid) sorted[s_base + s_warp[warp] + __popc(mask & ((1u << lane) - 1u))] = make_uint2((uint32_t)i, s);
        __syncthreads();
    }
}

// The paper's SABA arrangement for the literal SABA word: inside each start
// vertex's bucket, walks ordered by their seed X_W (the low 32 bits of the
// walk key; ties by id), so that a bouquet holds walks whose seeds, and so
// whose first choices, are close.  One block per bucket, a bitonic sort in
// shared memory of runs of up to kSabaRun walks (longer buckets are ordered
// run by run).  The order changes which walks share a warp, not any result.
constexpr uint32_t kSabaRun = 1024;

__global__ void __launch_bounds__(256)
saba_order_kernel(const uint32_t *__restrict__ counts, const uint32_t *__restrict__ cursor, uint32_t n,
                  uint64_t seed, uint2 *__restrict__ sorted) {
    __shared__ uint32_t s_key[kSabaRun];
    __shared__ uint32_t s_id[kSabaRun];
    for (uint32_t v = blockIdx.x; v < n; v += gridDim.x) {
        const uint32_t c = counts[v];
        if (c < 2) continue;
        const uint32_t end = cursor[v];  // after the scatter: one past v's bucket
        for (uint32_t lo = end - c; lo < end; lo += kSabaRun) {
            const uint32_t len = end - lo < kSabaRun ? end - lo : kSabaRun;
            uint32_t m = 2;
            while (m < len) m <<= 1;
            for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
                if (i < len) {
                    const uint32_t id = sorted[lo + i].x;
                    s_id[i] = id;
                    s_key[i] = (uint32_t)walk_key(seed, kBatchStream, id);
                } else {
                    s_id[i] = 0xffffffffu;
                    s_key[i] = 0xffffffffu;
                }
            }
            __syncthreads();
            for (uint32_t k = 2; k <= m; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
                        const uint32_t p = i ^ j;
                        if (p > i) {
                            const bool up = (i & k) == 0;
                            const uint64_t a = ((uint64_t)s_key[i] << 32) | s_id[i];
                            const uint64_t b = ((uint64_t)s_key[p] << 32) | s_id[p];
                            if ((a > b) == up) {
                                s_key[i] = (uint32_t)(b >> 32);
                                s_id[i] = (uint32_t)b;
                                s_key[p] = (uint32_t)(a >> 32);
                                s_id[p] = (uint32_t)a;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) sorted[lo + i].x = s_id[i];
            __syncthreads();
        }
    }
}

// -------------------------------------------------------------- bouquet

// Warp w owns grouped slots [w * 32 * W, (w + 1) * 32 * W); slot j of lane l
// is position w*32*W + j*32 + l, so each of the W lockstep groups is 32
// consecutive walks of the grouped order (a bouquet: mostly one start
// vertex).  Each lane advances W independent walks per step, keeping W
// dependent gather chains in flight per thread.  A walk carries (vertex, row
// offset, degree) from step to step, so with edge records a step is a single
// dependent load.  With `agg`, lanes standing on the same vertex merge their
// visit increments (match + popc) before one atomic.
template <typename EL, int W, bool COUPLED>
__global__ void __launch_bounds__(kThreads)
walk_bouquet_kernel(EL el, const int64_t *__restrict__ offsets, const uint2 *__restrict__ sorted, const uint32_t *__restrict__ n_valid_ptr,
                    uint32_t n_steps, uint64_t seed, Sampler smp, bool visit_start, bool checked, bool agg,
                    uint32_t *__restrict__ visits, uint32_t *__restrict__ paths, uint32_t *status) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_valid = *n_valid_ptr;
    const uint64_t base = warp * 32ull * W;
    if (base >= n_valid) return;

    uint32_t cur[W], id[W], deg[W], amask[W];
    uint64_t off[W], st[W], gs[W];
    uint32_t xw[W];  // the walk's fixed seed (literal SABA word only)
    bool act[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const uint64_t p = base + (uint64_t)j * 32 + lane;
        act[j] = p < n_valid;
        amask[j] = __ballot_sync(0xffffffffu, act[j]);
        const uint2 ws = act[j] ? sorted[p] : make_uint2(0u, 0u);
        id[j] = ws.x;
        cur[j] = ws.y;
        off[j] = 0;
        deg[j] = 0;
        if (act[j]) start_record(offsets, cur[j], off[j], deg[j]);
        st[j] = walk_key(seed, kBatchStream, id[j]);
        gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, smp.t == kSabaT ? 0 : id[j] / smp.width)
                        : 0ull;
        xw[j] = (uint32_t)st[j];
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (!act[j]) continue;
        if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = cur[j];
        if (visit_start) {
            if (agg) {
                const uint32_t peers = __match_any_sync(amask[j], cur[j]);
                if (lane == (uint32_t)(__ffs(peers) - 1)) add_visits(visits, cur[j], __popc(peers), checked, status);
            } else {
                add_visits(visits, cur[j], 1, checked, status);
            }
        }
    }
    for (uint32_t l = 1; l <= n_steps; ++l) {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            st[j] += kGolden;
            if (COUPLED) gs[j] += kGolden;
            if (deg[j]) {
                const uint32_t k = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t, xw[j]), deg[j]);
                el.next(off[j] + k, cur[j], off[j], deg[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (!act[j]) continue;
            if (agg) {
                const uint32_t peers = __match_any_sync(amask[j], cur[j]);
                if (lane == (uint32_t)(__ffs(peers) - 1)) add_visits(visits, cur[j], __popc(peers), checked, status);
            } else {
                add_visits(visits, cur[j], 1, checked, status);
            }
            if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = cur[j];
        }
    }
}

// The bouquet walk with a shared-memory hub table.  The random walk stands on
// a vertex in proportion to its degree, so the few highest-degree vertices
// receive a large share of all visits (39% for 8192 slots on R-MAT scale 20).
// Each block copies the graph's hub table (slot -> vertex) and those
// vertices' records into shared memory; a step landing on a hub reads the
// record and adds the visit there instead of in global memory, which removes
// two of the three global sector accesses of that step.  The block's hub
// counts are added to `visits` when it finishes.  The grid is persistent
// (one block per SM at 1024 threads): warps pull chunks of 32*W grouped walks
// from a counter, so the table is filled once per block.
constexpr int kHubThreads = 1024;

template <typename EL, int W, bool COUPLED>
__global__ void __launch_bounds__(kHubThreads, 1)
walk_hub_kernel(EL el, const int64_t *__restrict__ offsets, const uint32_t *__restrict__ hub_tag, uint32_t hub_slots,
                const uint2 *__restrict__ sorted,
                const uint32_t *__restrict__ n_valid_ptr, uint32_t n_steps, uint64_t seed, Sampler smp,
                bool visit_start, uint32_t *__restrict__ visits, uint32_t *__restrict__ paths,
                unsigned long long *__restrict__ next_chunk, bool l2_hints) {
    extern __shared__ __align__(16) unsigned char hub_smem[];
    const uint64_t pol_keep = l2_hints ? l2_policy_keep() : 0ull;
    const uint64_t pol_stream = l2_hints ? l2_policy_stream() : 0ull;
    const uint32_t slots = hub_slots;
    uint2 *s_rec = reinterpret_cast<uint2 *>(hub_smem);
    uint32_t *s_tag = reinterpret_cast<uint32_t *>(s_rec + slots);
    uint32_t *s_cnt = s_tag + slots;
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const uint32_t t = hub_tag[i];
        s_tag[i] = t;
        s_cnt[i] = 0;
        uint2 r = make_uint2(0u, 0u);
        if constexpr (EL::kSplit) {
            if (t != kNoHub) {
                uint64_t o;
                uint32_t d;
                el.rec_of(t, o, d);
                r = make_uint2((uint32_t)o, d);
            }
        }
        s_rec[i] = r;
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n_valid = *n_valid_ptr;
    while (true) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint64_t base = chunk * 32ull * W;
        if (base >= n_valid) break;

        uint32_t cur[W], id[W], deg[W];
        uint64_t off[W], st[W], gs[W];
        uint32_t xw[W];  // the walk's fixed seed (literal SABA word only)
        bool act[W], moved[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t p = base + (uint64_t)j * 32 + lane;
            act[j] = p < n_valid;
            id[j] = 0u;
            cur[j] = 0u;
            if (act[j]) {
                const uint2 ws = l2_hints ? ldg_pol(sorted + p, pol_stream) : sorted[p];
                id[j] = ws.x;
                cur[j] = ws.y;
            }
            off[j] = 0;
            deg[j] = 0;
            if (act[j]) start_record(offsets, cur[j], off[j], deg[j]);
            st[j] = walk_key(seed, kBatchStream, id[j]);
            gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, smp.t == kSabaT ? 0 : id[j] / smp.width)
                            : 0ull;
            xw[j] = (uint32_t)st[j];
            if (act[j]) {
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = cur[j];
                if (visit_start) {
                    const uint32_t slot = hub_slot(cur[j], slots);
                    if (s_tag[slot] == cur[j]) atomicAdd(s_cnt + slot, 1u);
                    else atomicAdd(visits + cur[j], 1u);
                }
            }
        }
        for (uint32_t l = 1; l <= n_steps; ++l) {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                st[j] += kGolden;
                if (COUPLED) gs[j] += kGolden;
                moved[j] = deg[j] != 0;
                if (moved[j]) {
                    const uint32_t k = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t, xw[j]), deg[j]);
                    if constexpr (EL::kSplit) cur[j] = l2_hints ? el.id(off[j] + k, pol_keep) : el.id(off[j] + k);
                    else el.next(off[j] + k, cur[j], off[j], deg[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (!act[j]) continue;
                const uint32_t slot = hub_slot(cur[j], slots);
                if (s_tag[slot] == cur[j]) {
                    atomicAdd(s_cnt + slot, 1u);
                    if constexpr (EL::kSplit) {
                        if (moved[j]) {
                            const uint2 r = s_rec[slot];
                            off[j] = r.x;
                            deg[j] = r.y;
                        }
                    }
                } else {
                    atomicAdd(visits + cur[j], 1u);
                    if constexpr (EL::kSplit) {
                        if (moved[j]) {
                            if (l2_hints) el.rec_of(cur[j], off[j], deg[j], pol_keep);
                            else el.rec_of(cur[j], off[j], deg[j]);
                        }
                    }
                }
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = cur[j];
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        if (c) atomicAdd(visits + s_tag[i], c);
    }
}

// The hub table spread over a thread-block cluster: CTA r of a cluster of C
// holds slots [r * per, (r + 1) * per) of a table of C * per slots, so a
// cluster covers C times the hubs of one CTA with the same shared memory per
// CTA (and so the same L1 left for the walks' gathers).  A step reads its
// vertex's slot in the owning CTA through distributed shared memory and adds
// a hub visit there.  The cluster synchronises once the slices are filled
// and again before any CTA flushes its counts and exits, so no CTA touches
// the shared memory of a CTA that has left.
template <typename EL, int W, bool COUPLED>
__global__ void __launch_bounds__(kHubThreads, 1)
walk_cluster_hub_kernel(EL el, const int64_t *__restrict__ offsets, const uint32_t *__restrict__ hub_tag,
                        uint32_t hub_slots, const uint2 *__restrict__ sorted, const uint32_t *__restrict__ n_valid_ptr,
                        uint32_t n_steps, uint64_t seed, Sampler smp, bool visit_start,
                        uint32_t *__restrict__ visits, uint32_t *__restrict__ paths,
                        unsigned long long *__restrict__ next_chunk) {
    extern __shared__ __align__(16) unsigned char hub_smem[];
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t csize = cluster.num_blocks();
    const uint32_t rank = cluster.block_rank();
    const uint32_t per = hub_slots / csize;
    uint2 *s_rec = reinterpret_cast<uint2 *>(hub_smem);
    uint32_t *s_tag = reinterpret_cast<uint32_t *>(s_rec + per);
    uint32_t *s_cnt = s_tag + per;
    for (uint32_t i = threadIdx.x; i < per; i += blockDim.x) {
        const uint32_t t = hub_tag[rank * per + i];
        s_tag[i] = t;
        s_cnt[i] = 0;
        uint2 r = make_uint2(0u, 0u);
        if constexpr (EL::kSplit) {
            if (t != kNoHub) {
                uint64_t o;
                uint32_t d;
                el.rec_of(t, o, d);
                r = make_uint2((uint32_t)o, d);
            }
        }
        s_rec[i] = r;
    }
    cluster.sync();

    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n_valid = *n_valid_ptr;
    while (true) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint64_t base = chunk * 32ull * W;
        if (base >= n_valid) break;

        uint32_t cur[W], id[W], deg[W];
        uint64_t off[W], st[W], gs[W];
        uint32_t xw[W];  // the walk's fixed seed (literal SABA word only)
        bool act[W], moved[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t p = base + (uint64_t)j * 32 + lane;
            act[j] = p < n_valid;
            id[j] = 0u;
            cur[j] = 0u;
            if (act[j]) {
                const uint2 ws = sorted[p];
                id[j] = ws.x;
                cur[j] = ws.y;
            }
            off[j] = 0;
            deg[j] = 0;
            if (act[j]) start_record(offsets, cur[j], off[j], deg[j]);
            st[j] = walk_key(seed, kBatchStream, id[j]);
            gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, smp.t == kSabaT ? 0 : id[j] / smp.width)
                            : 0ull;
            xw[j] = (uint32_t)st[j];
            if (act[j]) {
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = cur[j];
                if (visit_start) {
                    const uint32_t slot = hub_slot(cur[j], hub_slots);
                    const uint32_t owner = slot / per, local = slot - owner * per;
                    if (cluster.map_shared_rank(s_tag, owner)[local] == cur[j])
                        atomicAdd(cluster.map_shared_rank(s_cnt, owner) + local, 1u);
                    else
                        atomicAdd(visits + cur[j], 1u);
                }
            }
        }
        for (uint32_t l = 1; l <= n_steps; ++l) {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                st[j] += kGolden;
                if (COUPLED) gs[j] += kGolden;
                moved[j] = deg[j] != 0;
                if (moved[j]) {
                    const uint32_t k = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t, xw[j]), deg[j]);
                    if constexpr (EL::kSplit) cur[j] = el.id(off[j] + k);
                    else el.next(off[j] + k, cur[j], off[j], deg[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (!act[j]) continue;
                const uint32_t slot = hub_slot(cur[j], hub_slots);
                const uint32_t owner = slot / per, local = slot - owner * per;
                if (cluster.map_shared_rank(s_tag, owner)[local] == cur[j]) {
                    atomicAdd(cluster.map_shared_rank(s_cnt, owner) + local, 1u);
                    if constexpr (EL::kSplit) {
                        if (moved[j]) {
                            const uint2 r = cluster.map_shared_rank(s_rec, owner)[local];
                            off[j] = r.x;
                            deg[j] = r.y;
                        }
                    }
                } else {
                    atomicAdd(visits + cur[j], 1u);
                    if constexpr (EL::kSplit) {
                        if (moved[j]) el.rec_of(cur[j], off[j], deg[j]);
                    }
                }
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = cur[j];
            }
        }
    }
    cluster.sync();
    for (uint32_t i = threadIdx.x; i < per; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        if (c) atomicAdd(visits + s_tag[i], c);
    }
}

// The bouquet walk on the degree-relabelled copy: internal ids 0..hubs-1
// are the highest-degree vertices, so a step finds a hub by comparing its
// internal id, with no hash and no tag.  Shared memory holds, per hub, its
// row offset (the next hub's offset ends the row), original id and visit
// count, 12 bytes; any other vertex's 16-byte record gives its row offset,
// degree and original id, packed into 8 bytes.  The step word is drawn at the original id, and
// rows keep their neighbour order, so every walk is the one the plain
// kernels take.  Visits go to the original ids.
template <int W, bool COUPLED>
__global__ void __launch_bounds__(kHubThreads, 1)
walk_relabel_kernel(EdgesPackedIds el, const uint4 *__restrict__ rl_rec, const uint64_t *__restrict__ rl_rec8,
                    uint32_t sh_off, uint32_t sh_deg, uint32_t mask_id, uint64_t mask_off,
                    const uint32_t *__restrict__ rl_new,
                    uint32_t hubs, const uint2 *__restrict__ sorted,
                    const uint32_t *__restrict__ n_valid_ptr, uint32_t n_steps, uint64_t seed, Sampler smp,
                    bool visit_start, uint32_t *__restrict__ visits, uint32_t *__restrict__ paths,
                    unsigned long long *__restrict__ next_chunk) {
    extern __shared__ __align__(16) unsigned char hub_smem[];
    uint32_t *s_off = reinterpret_cast<uint32_t *>(hub_smem);  // hubs + 1
    uint32_t *s_orig = s_off + hubs + 1;
    uint32_t *s_cnt = s_orig + hubs;
    for (uint32_t i = threadIdx.x; i < hubs; i += blockDim.x) {
        const uint4 r = rl_rec[i];
        s_off[i] = r.x;
        s_orig[i] = r.z;
        s_cnt[i] = 0;
        if (i == hubs - 1) s_off[hubs] = r.x + r.y;
    }
    __syncthreads();

    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n_valid = *n_valid_ptr;
    while (true) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint64_t base = chunk * 32ull * W;
        if (base >= n_valid) break;

        uint32_t x[W], orig[W], id[W], deg[W];
        uint64_t off[W], st[W], gs[W];
        uint32_t xw[W];  // the walk's fixed seed (literal SABA word only)
        bool act[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t p = base + (uint64_t)j * 32 + lane;
            act[j] = p < n_valid;
            id[j] = 0u;
            orig[j] = 0u;
            x[j] = 0u;
            off[j] = 0;
            deg[j] = 0;
            if (act[j]) {
                const uint2 ws = sorted[p];
                id[j] = ws.x;
                orig[j] = ws.y;
                x[j] = rl_new[orig[j]];
                if (x[j] < hubs) {
                    off[j] = s_off[x[j]];
                    deg[j] = s_off[x[j] + 1] - s_off[x[j]];
                } else {
                    const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(rl_rec8) + x[j]);
                    off[j] = (w >> sh_off) & mask_off;
                    deg[j] = (uint32_t)(w >> sh_deg);
                }
            }
            st[j] = walk_key(seed, kBatchStream, id[j]);
            gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, smp.t == kSabaT ? 0 : id[j] / smp.width)
                            : 0ull;
            xw[j] = (uint32_t)st[j];
            if (act[j]) {
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = orig[j];
                if (visit_start) {
                    if (x[j] < hubs) atomicAdd(s_cnt + x[j], 1u);
                    else atomicAdd(visits + orig[j], 1u);
                }
            }
        }
        for (uint32_t l = 1; l <= n_steps; ++l) {
            bool moved[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                st[j] += kGolden;
                if (COUPLED) gs[j] += kGolden;
                moved[j] = deg[j] != 0;
                if (moved[j]) {
                    const uint32_t k = choose(sample_word<COUPLED>(st[j], gs[j], orig[j], smp.t, xw[j]), deg[j]);
                    x[j] = el.id(off[j] + k);
                }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (!act[j]) continue;
                if (x[j] < hubs) {
                    atomicAdd(s_cnt + x[j], 1u);
                    if (moved[j]) {
                        off[j] = s_off[x[j]];
                        deg[j] = s_off[x[j] + 1] - s_off[x[j]];
                        orig[j] = s_orig[x[j]];
                    }
                } else {
                    if (moved[j]) {
                        const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(rl_rec8) + x[j]);
                        off[j] = (w >> sh_off) & mask_off;
                        deg[j] = (uint32_t)(w >> sh_deg);
                        orig[j] = (uint32_t)w & mask_id;
                    }
                    atomicAdd(visits + orig[j], 1u);
                }
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = orig[j];
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < hubs; i += blockDim.x) {
        const uint32_t c = s_cnt[i];
        if (c) atomicAdd(visits + s_orig[i], c);
    }
}

// The bouquet walk on the degree-relabelled copy with 8-byte shared-memory
// hubs.  Internal ids follow the degree order, so the first `hubs` of them
// are the highest-degree vertices, the number chosen at launch from the
// shared memory the plain relabel kernel's 12-byte entries take (16,383
// instead of 10,922 on R-MAT scale 20: 57 % of the visits instead of 49 %).
// A hub keeps its row offset (32 bits; the next hub's offset ends its row)
// and one 32-bit word {original id | count << cnt_shift}: a step to a hub is
// one 32-bit shared-memory atomic add of 1 << cnt_shift, which returns the
// original id and counts the visit.  The count field holds the bits above
// the id; when an add wraps it (the returned count is all ones) the walker
// adds 2^(32 - cnt_shift) to the vertex's visits, so no visit is lost.  Any
// other vertex reads its 8-byte record and adds its visit in L2, as in the
// plain kernel.  Each block adds its hub counts to the visits at the end.
// Paths and visits are those of every other walk kernel.
struct Hub8Fields {
    uint32_t sh_off;     // bits of the original id in a record
    uint32_t sh_deg;     // + bits of the row offset
    uint32_t mask_id;
    uint64_t mask_off;
    uint32_t mask_deg;
    uint32_t hubs;       // internal ids below this are served from shared memory
    uint32_t cnt_shift;  // a hub word's count field is bits [cnt_shift, 32)
    uint32_t n;
    uint64_t nnz;
};

template <int W, bool COUPLED>
__global__ void __launch_bounds__(kHubThreads, 1)
walk_relabel8_kernel(EdgesPackedIds el, const uint64_t *__restrict__ rl_rec8, Hub8Fields f,
                 const uint32_t *__restrict__ rl_new, const uint2 *__restrict__ sorted, const uint32_t *__restrict__ n_valid_ptr, uint32_t n_steps,
                 uint64_t seed, Sampler smp, bool visit_start, uint32_t *__restrict__ visits,
                 uint32_t *__restrict__ paths, unsigned long long *__restrict__ next_chunk) {
    extern __shared__ __align__(16) unsigned char hub_smem[];
    uint32_t *s_off = reinterpret_cast<uint32_t *>(hub_smem);  // hubs + 1 row offsets
    uint32_t *s_idc = s_off + f.hubs + 1;                      // hubs words {id | count}
    for (uint32_t i = threadIdx.x; i < f.hubs; i += blockDim.x) {
        const uint64_t w = __ldg(rl_rec8 + i);
        s_off[i] = (uint32_t)((w >> f.sh_off) & f.mask_off);
        s_idc[i] = (uint32_t)w & f.mask_id;
    }
    if (threadIdx.x == 0)  // the row end of the last hub
        s_off[f.hubs] = (uint32_t)(f.hubs < f.n ? (__ldg(rl_rec8 + f.hubs) >> f.sh_off) & f.mask_off : f.nnz);
    __syncthreads();
    const uint32_t one = 1u << f.cnt_shift, cmask = 0xffffffffu >> f.cnt_shift;

    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n_valid = *n_valid_ptr;
    while (true) {
        unsigned long long chunk = 0;
        if (lane == 0) chunk = atomicAdd(next_chunk, 1ull);
        chunk = __shfl_sync(0xffffffffu, chunk, 0);
        const uint64_t base = chunk * 32ull * W;
        if (base >= n_valid) break;

        uint32_t x[W], orig[W], id[W], deg[W], off[W];
        uint64_t st[W], gs[W];
        uint32_t xw[W];  // the walk's fixed seed (literal SABA word only)
        bool act[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t p = base + (uint64_t)j * 32 + lane;
            act[j] = p < n_valid;
            id[j] = 0u;
            orig[j] = 0u;
            x[j] = 0u;
            off[j] = 0u;
            deg[j] = 0u;
            if (act[j]) {
                const uint2 ws = sorted[p];
                id[j] = ws.x;
                orig[j] = ws.y;
                x[j] = rl_new[orig[j]];
                if (x[j] < f.hubs) {
                    if (visit_start) {
                        const uint32_t w = atomicAdd(s_idc + x[j], one);
                        if ((w >> f.cnt_shift) == cmask) atomicAdd(visits + orig[j], cmask + 1u);
                    }
                    off[j] = s_off[x[j]];
                    deg[j] = s_off[x[j] + 1] - off[j];
                } else {
                    const uint64_t w = __ldg(rl_rec8 + x[j]);
                    off[j] = (uint32_t)((w >> f.sh_off) & f.mask_off);
                    deg[j] = (uint32_t)(w >> f.sh_deg) & f.mask_deg;
                    if (visit_start) atomicAdd(visits + orig[j], 1u);
                }
            }
            st[j] = walk_key(seed, kBatchStream, id[j]);
            gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, smp.t == kSabaT ? 0 : id[j] / smp.width)
                            : 0ull;
            xw[j] = (uint32_t)st[j];
            if (act[j] && paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = orig[j];
        }
        for (uint32_t l = 1; l <= n_steps; ++l) {
            bool moved[W];
#pragma unroll
            for (int j = 0; j < W; ++j) {
                st[j] += kGolden;
                if (COUPLED) gs[j] += kGolden;
                moved[j] = deg[j] != 0;
                if (moved[j]) {
                    const uint32_t k = choose(sample_word<COUPLED>(st[j], gs[j], orig[j], smp.t, xw[j]), deg[j]);
                    x[j] = el.id((uint64_t)off[j] + k);
                }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
                if (!act[j]) continue;
                if (x[j] < f.hubs) {
                    const uint32_t w = atomicAdd(s_idc + x[j], one);
                    if ((w >> f.cnt_shift) == cmask) atomicAdd(visits + (w & f.mask_id), cmask + 1u);
                    if (moved[j]) {
                        orig[j] = w & f.mask_id;
                        off[j] = s_off[x[j]];
                        deg[j] = s_off[x[j] + 1] - off[j];
                    }
                } else {
                    if (moved[j]) {
                        const uint64_t w = __ldg(rl_rec8 + x[j]);
                        orig[j] = (uint32_t)w & f.mask_id;
                        off[j] = (uint32_t)((w >> f.sh_off) & f.mask_off);
                        deg[j] = (uint32_t)(w >> f.sh_deg) & f.mask_deg;
                    }
                    atomicAdd(visits + orig[j], 1u);
                }
                if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = orig[j];
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < f.hubs; i += blockDim.x) {
        const uint32_t w = s_idc[i];
        if (w >> f.cnt_shift) atomicAdd(visits + (w & f.mask_id), w >> f.cnt_shift);
    }
}

unsigned blocks_for(uint64_t items, uint64_t per_block) {
    uint64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 0x7fffffffull) b = 0x7fffffffull;
    return (unsigned)b;
}

template <typename RL>
int launch_naive(RL rl, const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                 uint32_t n_steps, const Sampler &smp, bool visit_start, bool checked, uint32_t *visits,
                 uint32_t *paths, uint32_t *status, cudaStream_t s) {
    const unsigned grid = blocks_for(n_walks, kThreads);
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    count_walk_kernel(BQ_WALK_KERNEL_NAIVE);
    if (smp.kind == 1)
        walk_naive_kernel<RL, true><<<grid, kThreads, 0, s>>>(rl, g.nbrs, g.n, starts, n_walks, n_steps, seed,
                                                              smp, visit_start, checked, visits, paths, status);
    else
        walk_naive_kernel<RL, false><<<grid, kThreads, 0, s>>>(rl, g.nbrs, g.n, starts, n_walks, n_steps, seed,
                                                               smp, visit_start, checked, visits, paths, status);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

template <typename EL, int W>
void launch_bouquet_w(EL el, const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                      uint64_t n_walks, uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start,
                      bool checked, bool agg, uint32_t *visits, uint32_t *paths, uint32_t *status, cudaStream_t s) {
    const unsigned grid = blocks_for(n_walks, (uint64_t)kThreads * W);
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    count_walk_kernel(BQ_WALK_KERNEL_BOUQUET);
    if (smp.kind == 1)
        walk_bouquet_kernel<EL, W, true><<<grid, kThreads, 0, s>>>(el, g.offsets, sorted, n_valid, n_steps, seed,
                                                                   smp, visit_start, checked, agg, visits, paths,
                                                                   status);
    else
        walk_bouquet_kernel<EL, W, false><<<grid, kThreads, 0, s>>>(el, g.offsets, sorted, n_valid, n_steps, seed,
                                                                    smp, visit_start, checked, agg, visits, paths,
                                                                    status);
}

template <typename EL>
void launch_bouquet_any(EL el, const DeviceGraph &g, const uint2 *sorted,
                        const uint32_t *n_valid, uint64_t n_walks, uint32_t n_steps, uint64_t seed,
                        const Sampler &smp, bool visit_start, bool checked, bool agg, uint32_t *visits,
                        uint32_t *paths, uint32_t *status, int lanes_w, cudaStream_t s) {
    switch (lanes_w) {
    case 1: launch_bouquet_w<EL, 1>(el, g, sorted, n_valid, n_walks, n_steps, seed, smp, visit_start, checked, agg,
                                    visits, paths, status, s); break;
    case 2: launch_bouquet_w<EL, 2>(el, g, sorted, n_valid, n_walks, n_steps, seed, smp, visit_start, checked, agg,
                                    visits, paths, status, s); break;
    case 8: launch_bouquet_w<EL, 8>(el, g, sorted, n_valid, n_walks, n_steps, seed, smp, visit_start, checked, agg,
                                    visits, paths, status, s); break;
    default: launch_bouquet_w<EL, 4>(el, g, sorted, n_valid, n_walks, n_steps, seed, smp, visit_start, checked,
                                     agg, visits, paths, status, s); break;
    }
}

// Launch the hub kernel; returns false (nothing launched) when a block of
// kHubThreads with the table does not fit on an SM.
template <typename EL, int W, bool COUPLED>
bool launch_hub_w(EL el, const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                  uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                  uint32_t *paths, unsigned long long *next_chunk, cudaStream_t s) {
    const size_t smem = (size_t)16 * g.hub_slots;
    auto kernel = walk_hub_kernel<EL, W, COUPLED>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kHubThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    count_walk_kernel(BQ_WALK_KERNEL_HUB);
    kernel<<<sms * per_sm, kHubThreads, smem, s>>>(el, g.offsets, g.hub_tag, g.hub_slots, sorted, n_valid, n_steps,
                                                   seed, smp, visit_start, visits, paths, next_chunk,
                                                   tuning_l2_hints());
    return true;
}

template <typename EL>
bool launch_hub(EL el, const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                uint32_t *paths, unsigned long long *next_chunk, int lanes_w, cudaStream_t s) {
    const bool c = smp.kind == 1;
#define BQ_HUB(WW)                                                                                                 \
    (c ? launch_hub_w<EL, WW, true>(el, g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,   \
                                    next_chunk, s)                                                             \
       : launch_hub_w<EL, WW, false>(el, g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,  \
                                     next_chunk, s))
    if (lanes_w == 1) return BQ_HUB(1);
    if (lanes_w == 2) return BQ_HUB(2);
    return BQ_HUB(4);
#undef BQ_HUB
}

// Launch the cluster hub kernel: clusters of g.hub_cluster CTAs, as many as
// can be resident at once (the grid is persistent); false (nothing launched)
// when no such cluster fits.
template <typename EL, int W, bool COUPLED>
bool launch_cluster_hub_w(EL el, const DeviceGraph &g, const uint2 *sorted,
                          const uint32_t *n_valid, uint32_t n_steps, uint64_t seed, const Sampler &smp,
                          bool visit_start, uint32_t *visits, uint32_t *paths, unsigned long long *next_chunk,
                          cudaStream_t s) {
    const uint32_t csize = g.hub_cluster;
    const size_t smem = (size_t)16 * (g.hub_slots / csize);
    auto kernel = walk_cluster_hub_kernel<EL, W, COUPLED>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(kHubThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg) != cudaSuccess || clusters < 1) {
        cudaGetLastError();
        return false;
    }
    cfg.gridDim = dim3((unsigned)clusters * csize);
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    if (cudaLaunchKernelEx(&cfg, kernel, el, g.offsets, g.hub_tag, g.hub_slots, sorted, n_valid, n_steps, seed, smp,
                           visit_start, visits, paths, next_chunk) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    count_walk_kernel(BQ_WALK_KERNEL_CLUSTER_HUB);
    return true;
}

template <typename EL>
bool launch_cluster_hub(EL el, const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                        uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                        uint32_t *paths, unsigned long long *next_chunk, int lanes_w, cudaStream_t s) {
    const bool c = smp.kind == 1;
#define BQ_CHUB(WW)                                                                                             \
    (c ? launch_cluster_hub_w<EL, WW, true>(el, g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, \
                                            paths, next_chunk, s)                                             \
       : launch_cluster_hub_w<EL, WW, false>(el, g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, \
                                             paths, next_chunk, s))
    if (lanes_w == 1) return BQ_CHUB(1);
    if (lanes_w == 2) return BQ_CHUB(2);
    return BQ_CHUB(4);
#undef BQ_CHUB
}

// Launch the relabelled-copy kernel: one persistent block of kHubThreads per
// SM; false (nothing launched) when the hub arrays do not fit.
template <int W, bool COUPLED>
bool launch_relabel_w(const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                      uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                      uint32_t *paths, unsigned long long *next_chunk, cudaStream_t s) {
    const size_t smem = (size_t)12 * g.rl_hubs + 4;
    auto kernel = walk_relabel_kernel<W, COUPLED>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kHubThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    const EdgesPackedIds el{g.rl_pk, nullptr, g.pk_bits, g.pk_q, g.pk_mask};
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    count_walk_kernel(BQ_WALK_KERNEL_RELABEL);
    kernel<<<sms * per_sm, kHubThreads, smem, s>>>(el, g.rl_rec, g.rl_rec8, g.rl_sh_off, g.rl_sh_deg, g.rl_mask_id,
                                                   g.rl_mask_off, g.rl_new, g.rl_hubs, sorted, n_valid, n_steps,
                                                   seed, smp, visit_start, visits, paths, next_chunk);
    return true;
}

bool launch_relabel(const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                    uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                    uint32_t *paths, unsigned long long *next_chunk, int lanes_w, cudaStream_t s) {
    const bool c = smp.kind == 1;
#define BQ_RL(WW)                                                                                               \
    (c ? launch_relabel_w<WW, true>(g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,        \
                                    next_chunk, s)                                                               \
       : launch_relabel_w<WW, false>(g, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,       \
                                     next_chunk, s))
    if (lanes_w == 1) return BQ_RL(1);
    if (lanes_w == 2) return BQ_RL(2);
    return BQ_RL(4);
#undef BQ_RL
}

// The 8-byte-hub kernel's fields on this graph, and whether it can run: the
// hubs must cover every vertex whose degree the records do not hold, row
// offsets must fit 32 bits, and a hub word needs at least kMinCountBits
// count bits above the id.
constexpr uint32_t kMinCountBits = 8;

bool hub8_fields(const DeviceGraph &g, Hub8Fields &f) {
    if (!g.rl_pk || !g.rl_rec8 || g.nnz >= (1ull << 32) || g.rl_sh_off >= 32) return false;
    uint32_t hubs = tuning_hub8_hubs();
    if (hubs == 0)  // as many as the plain relabel kernel's shared memory holds
        hubs = (uint32_t)(((size_t)12 * g.rl_hubs + 4 - 4) / 8);
    if (hubs > g.rl_live) hubs = g.rl_live;
    if (hubs < g.rl_fit) return false;
    const uint32_t cap = tuning_hub8_count_bits();
    uint32_t bits = 32 - g.rl_sh_off;
    if (bits < kMinCountBits && !cap) return false;
    if (cap && cap < bits) bits = cap;
    f.sh_off = g.rl_sh_off;
    f.sh_deg = g.rl_sh_deg;
    f.mask_id = g.rl_mask_id;
    f.mask_off = g.rl_mask_off;
    f.mask_deg = g.rl_bits_deg >= 32 ? 0xffffffffu : ((1u << g.rl_bits_deg) - 1u);
    f.hubs = hubs;
    f.cnt_shift = 32 - bits;
    f.n = g.n;
    f.nnz = g.nnz;
    return true;
}

template <int W, bool COUPLED>
bool launch_hub8_w(const DeviceGraph &g, const Hub8Fields &f, const uint2 *sorted,
                   const uint32_t *n_valid, uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start,
                   uint32_t *visits, uint32_t *paths, unsigned long long *next_chunk, cudaStream_t s) {
    const size_t smem = (size_t)8 * f.hubs + 4;
    auto kernel = walk_relabel8_kernel<W, COUPLED>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kHubThreads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    const EdgesPackedIds el{g.rl_pk, nullptr, g.pk_bits, g.pk_q, g.pk_mask};
    ProfScope prof(kProfWalk, s);
    count_launches(1);
    count_walk_kernel(BQ_WALK_KERNEL_RELABEL8);
    kernel<<<sms * per_sm, kHubThreads, smem, s>>>(el, g.rl_rec8, f, g.rl_new, sorted, n_valid, n_steps, seed, smp,
                                                   visit_start, visits, paths, next_chunk);
    return true;
}

bool launch_hub8(const DeviceGraph &g, const uint2 *sorted, const uint32_t *n_valid,
                 uint32_t n_steps, uint64_t seed, const Sampler &smp, bool visit_start, uint32_t *visits,
                 uint32_t *paths, unsigned long long *next_chunk, int lanes_w, cudaStream_t s) {
    Hub8Fields f;
    if (!tuning_relabel_hub8() || !hub8_fields(g, f)) return false;
    const bool c = smp.kind == 1;
#define BQ_H8(WW)                                                                                               \
    (c ? launch_hub8_w<WW, true>(g, f, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,       \
                                 next_chunk, s)                                                                   \
       : launch_hub8_w<WW, false>(g, f, sorted, n_valid, n_steps, seed, smp, visit_start, visits, paths,      \
                                  next_chunk, s))
    if (lanes_w == 1) return BQ_H8(1);
    if (lanes_w == 2) return BQ_H8(2);
    return BQ_H8(4);
#undef BQ_H8
}

// Group the walks by start vertex into `sorted` (walk id, start) pairs;
// cursor[n] = valid walks.
int group_by_start(const DeviceGraph &g, const uint32_t *starts, uint64_t n_walks, uint32_t *counts, uint32_t *cursor,
                   uint2 *sorted, uint32_t *status, void *scan_ws, size_t scan_ws_bytes,
                   cudaStream_t s) {
    BQ_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * g.n, s));
    const unsigned grid = blocks_for(n_walks, kThreads * 4);
    ProfScope prof(kProfGroup, s);
    count_launches(2);
    hist_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, counts, status);
    const int rc = scan_ws ? scan_u32_ws(counts, cursor, g.n, scan_ws, scan_ws_bytes, s)
                           : scan_u32(counts, cursor, g.n, s);
    if (rc) return rc;
    scatter_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, cursor, sorted);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

// counts[n] | cursor[n + 1] | (8-byte aligned) sorted (id, start) pairs |
// chunk counter
size_t bouquet_pairs_offset(uint32_t n) { return (sizeof(uint32_t) * (2 * (size_t)n + 1) + 7) & ~(size_t)7; }

size_t bouquet_counter_offset(uint32_t n, uint64_t n_walks) {
    return (bouquet_pairs_offset(n) + sizeof(uint2) * (size_t)n_walks + 15) & ~(size_t)15;
}

size_t bouquet_arrays_bytes(uint32_t n, uint64_t n_walks) {
    return (bouquet_counter_offset(n, n_walks) + 16 + 255) & ~(size_t)255;
}

// The bouquet walk batch in `scratch` (counts[n] | cursor[n + 1] | sorted
// ids | sorted starts, then the scan workspace when scan_ws is set).
int bouquet_in(const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks, uint32_t n_steps,
               const Sampler &smp, bool visit_start, uint32_t *visits, uint32_t *paths, uint32_t *status,
               char *scratch, char *scan_ws, size_t scan_ws_bytes, cudaStream_t s) {
    const uint64_t positions = (uint64_t)n_steps + (visit_start ? 1 : 0);
    // Below this bound a counter that starts at zero cannot wrap.
    const bool checked = positions > 0 && n_walks > 0xffffffffull / positions;
    const int lanes_w = tuning_walks_per_lane();
    const bool agg = tuning_aggregate_visits();
    const size_t n = g.n;
    uint32_t *counts = (uint32_t *)scratch, *cursor = counts + n;
    uint2 *sorted = reinterpret_cast<uint2 *>(scratch + bouquet_pairs_offset(g.n));
    const bool grouped = tuning_group_walks();
    int rc = BQ_OK;
    if (grouped) {
        rc = group_by_start(g, starts, n_walks, counts, cursor, sorted, status, scan_ws, scan_ws_bytes, s);
    } else {  // the same kernels on the walks in input order (cursor[n] = valid walks)
        BQ_CUDA(cudaMemsetAsync(cursor + n, 0, sizeof(uint32_t), s));
        ProfScope prof(kProfGroup, s);
        count_launches(1);
        pairs_in_order_kernel<<<blocks_for(n_walks, kPairTile), kPairTile, 0, s>>>(starts, n_walks, g.n, cursor + n,
                                                                                     sorted, status);
        BQ_CUDA(cudaGetLastError());
    }
    if (rc) return rc;
    if (grouped && smp.kind == 1 && smp.t == kSabaT) {
        ProfScope prof(kProfGroup, s);
        count_launches(1);
        int dev = 0, sms = 0;
        BQ_CUDA(cudaGetDevice(&dev));
        BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        saba_order_kernel<<<sms * 8, 256, 0, s>>>(counts, cursor, g.n, seed, sorted);
        BQ_CUDA(cudaGetLastError());
    }
    if (g.rl_pk && !checked) {
        auto *next_chunk = reinterpret_cast<unsigned long long *>(scratch + bouquet_counter_offset(g.n, n_walks));
        BQ_CUDA(cudaMemsetAsync(next_chunk, 0, sizeof(unsigned long long), s));
        if (launch_hub8(g, sorted, cursor + n, n_steps, seed, smp, visit_start, visits, paths, next_chunk,
                        lanes_w, s)) {
            BQ_CUDA(cudaGetLastError());
            return BQ_OK;
        }
        if (launch_relabel(g, sorted, cursor + n, n_steps, seed, smp, visit_start, visits, paths, next_chunk,
                           lanes_w, s)) {
            BQ_CUDA(cudaGetLastError());
            return BQ_OK;
        }
    }
    if (g.hub_tag && !checked) {
        auto *next_chunk = reinterpret_cast<unsigned long long *>(scratch + bouquet_counter_offset(g.n, n_walks));
        BQ_CUDA(cudaMemsetAsync(next_chunk, 0, sizeof(unsigned long long), s));
        const bool launched = with_edges(g, [&](auto el) {
            if (g.hub_cluster > 1)
                return launch_cluster_hub(el, g, sorted, cursor + n, n_steps, seed, smp, visit_start, visits,
                                          paths, next_chunk, lanes_w, s) ? 1 : 0;
            return launch_hub(el, g, sorted, cursor + n, n_steps, seed, smp, visit_start, visits, paths,
                              next_chunk, lanes_w, s) ? 1 : 0;
        });
        if (launched) {
            BQ_CUDA(cudaGetLastError());
            return BQ_OK;
        }
    }
    rc = with_edges(g, [&](auto el) {
        launch_bouquet_any(el, g, sorted, cursor + n, n_walks, n_steps, seed, smp, visit_start, checked, agg,
                           visits, paths, status, lanes_w, s);
        return BQ_OK;
    });
    BQ_CUDA(cudaGetLastError());
    return rc;
}

}  // namespace

size_t walk_batch_scratch_bytes(uint32_t n, uint64_t n_walks) {
    return bouquet_arrays_bytes(n, n_walks) + scan_u32_ws_bytes(n);
}

int launch_walk_batch_in(const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                         uint32_t n_steps, const Sampler &smp, bool visit_start, uint32_t *visits, uint32_t *paths,
                         uint32_t *status, void *scratch, size_t scratch_bytes, cudaStream_t s) {
    if (n_walks == 0) return BQ_OK;
    if (walk_batch_scratch_bytes(g.n, n_walks) > scratch_bytes) return fail(BQ_EINVAL, "scratch too small");
    const size_t arrays = bouquet_arrays_bytes(g.n, n_walks);
    char *base = (char *)scratch;
    return bouquet_in(g, seed, starts, n_walks, n_steps, smp, visit_start, visits, paths, status, base, base + arrays,
                      scratch_bytes - arrays, s);
}

int launch_walk_batch(const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                      uint32_t n_steps, uint32_t mode, const Sampler &smp, bool visit_start, uint32_t *visits,
                      uint32_t *paths, uint32_t *status, cudaStream_t s) {
    if (n_walks == 0) return BQ_OK;
    if (mode == BQ_MODE_NAIVE) {
        const uint64_t positions = (uint64_t)n_steps + (visit_start ? 1 : 0);
        const bool checked = positions > 0 && n_walks > 0xffffffffull / positions;
        if (g.compact())
            return launch_naive(RecCompact{g.rec8}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked,
                                visits, paths, status, s);
        return launch_naive(RecWide{g.rec16}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked, visits,
                            paths, status, s);
    }
    char *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, bouquet_arrays_bytes(g.n, n_walks), s);
    if (rc) return rc;
    rc = bouquet_in(g, seed, starts, n_walks, n_steps, smp, visit_start, visits, paths, status, buf, nullptr, 0, s);
    scratch_free(buf, s);
    return rc;
}

}  // namespace bq
