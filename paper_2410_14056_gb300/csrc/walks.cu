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
// Memory per step (the random gathers Sec. 3.2 names as the bottleneck):
// one vertex record {row offset, degree} (8 B, or 16 B for graphs with
// nnz >= 2^32) and one 4-byte neighbour id, plus a 4-byte visit atomic.
#include <algorithm>

#include "hash.cuh"
#include "internal.h"

namespace bq {
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
        uint64_t gs = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, i / smp.width) : 0;
        uint32_t *row = paths ? paths + i * ((uint64_t)n_steps + 1) : nullptr;
        if (row) row[0] = cur;
        if (visit_start) add_visits(visits, cur, 1, checked, status);
        for (uint32_t l = 1; l <= n_steps; ++l) {
            st += kGolden;
            if (COUPLED) gs += kGolden;
            uint64_t off;
            uint32_t d;
            rl.load(cur, off, d);
            if (d) cur = nbrs[off + choose(sample_word<COUPLED>(st, gs, cur, smp.t), d)];
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
                                      uint32_t *__restrict__ cursor, uint32_t *__restrict__ sorted_id,
                                      uint32_t *__restrict__ sorted_start) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_walks;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = starts[i];
        if (s >= n) continue;
        const uint32_t pos = atomicAdd(cursor + s, 1u);
        sorted_id[pos] = (uint32_t)i;
        sorted_start[pos] = s;
    }
}

// -------------------------------------------------------------- bouquet

// Warp w owns sorted slots [w * 32 * W, (w + 1) * 32 * W); slot j of lane l
// is position w*32*W + j*32 + l, so each of the W lockstep groups is 32
// consecutive walks of the grouped order (a bouquet: mostly one start
// vertex).  Each lane advances W independent walks per step, which keeps W
// dependent gather chains in flight per thread.  With AGG, lanes standing on
// the same vertex merge their visit increments (match + popc) before one
// atomic.
template <typename RL, int W, bool COUPLED, bool AGG>
__global__ void __launch_bounds__(kThreads)
walk_bouquet_kernel(RL rl, const uint32_t *__restrict__ nbrs, const uint32_t *__restrict__ sorted_id,
                    const uint32_t *__restrict__ sorted_start, const uint32_t *__restrict__ n_valid_ptr,
                    uint32_t n_steps, uint64_t seed, Sampler smp, bool visit_start, bool checked,
                    uint32_t *__restrict__ visits, uint32_t *__restrict__ paths, uint32_t *status) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_valid = *n_valid_ptr;
    const uint64_t base = warp * 32ull * W;
    if (base >= n_valid) return;

    uint32_t cur[W], id[W], amask[W];
    uint64_t st[W], gs[W];
    bool act[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        const uint64_t p = base + (uint64_t)j * 32 + lane;
        act[j] = p < n_valid;
        amask[j] = __ballot_sync(0xffffffffu, act[j]);
        id[j] = act[j] ? sorted_id[p] : 0u;
        cur[j] = act[j] ? sorted_start[p] : 0u;
        st[j] = walk_key(seed, kBatchStream, id[j]);
        gs[j] = COUPLED ? walk_key(seed, kBatchStream | kGroupBit, id[j] / smp.width) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if (paths && act[j]) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1)] = cur[j];
        if (visit_start && act[j]) {
            if (AGG) {
                const uint32_t peers = __match_any_sync(amask[j], cur[j]);
                if (lane == (uint32_t)(__ffs(peers) - 1)) add_visits(visits, cur[j], __popc(peers), checked, status);
            } else {
                add_visits(visits, cur[j], 1, checked, status);
            }
        }
    }
    for (uint32_t l = 1; l <= n_steps; ++l) {
        uint64_t off[W];
        uint32_t d[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            st[j] += kGolden;
            if (COUPLED) gs[j] += kGolden;
            d[j] = 0;
            off[j] = 0;
            if (act[j]) rl.load(cur[j], off[j], d[j]);
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (d[j]) cur[j] = nbrs[off[j] + choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), d[j])];
        }
#pragma unroll
        for (int j = 0; j < W; ++j) {
            if (!act[j]) continue;
            if (AGG) {
                const uint32_t peers = __match_any_sync(amask[j], cur[j]);
                if (lane == (uint32_t)(__ffs(peers) - 1)) add_visits(visits, cur[j], __popc(peers), checked, status);
            } else {
                add_visits(visits, cur[j], 1, checked, status);
            }
            if (paths) paths[(uint64_t)id[j] * ((uint64_t)n_steps + 1) + l] = cur[j];
        }
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
    if (smp.kind == 1)
        walk_naive_kernel<RL, true><<<grid, kThreads, 0, s>>>(rl, g.nbrs, g.n, starts, n_walks, n_steps, seed,
                                                              smp, visit_start, checked, visits, paths, status);
    else
        walk_naive_kernel<RL, false><<<grid, kThreads, 0, s>>>(rl, g.nbrs, g.n, starts, n_walks, n_steps, seed,
                                                               smp, visit_start, checked, visits, paths, status);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

template <typename RL, int W>
void launch_bouquet_w(RL rl, const DeviceGraph &g, const uint32_t *sid, const uint32_t *sst,
                      const uint32_t *n_valid, uint64_t n_walks, uint32_t n_steps, uint64_t seed,
                      const Sampler &smp, bool visit_start, bool checked, bool agg, uint32_t *visits,
                      uint32_t *paths, uint32_t *status, cudaStream_t s) {
    const unsigned grid = blocks_for(n_walks, (uint64_t)kThreads * W);
    ProfScope prof(kProfWalk, s);
    count_launches(1);
#define BQ_LAUNCH(C, A)                                                                                \
    walk_bouquet_kernel<RL, W, C, A><<<grid, kThreads, 0, s>>>(rl, g.nbrs, sid, sst, n_valid, n_steps, seed, \
                                                               smp, visit_start, checked, visits, paths, status)
    if (smp.kind == 1) {
        if (agg) BQ_LAUNCH(true, true);
        else BQ_LAUNCH(true, false);
    } else {
        if (agg) BQ_LAUNCH(false, true);
        else BQ_LAUNCH(false, false);
    }
#undef BQ_LAUNCH
}

template <typename RL>
int launch_bouquet(RL rl, const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                   uint32_t n_steps, const Sampler &smp, bool visit_start, bool checked, uint32_t *visits,
                   uint32_t *paths, uint32_t *status, int lanes_w, bool agg, cudaStream_t s) {
    // scratch: counts[n] | cursor[n + 1] | sorted_id[n_walks] | sorted_start[n_walks]
    const size_t n = g.n;
    const size_t bytes = sizeof(uint32_t) * (2 * n + 1 + 2 * (size_t)n_walks);
    uint32_t *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, bytes, s);
    if (rc) return rc;
    uint32_t *counts = buf, *cursor = buf + n, *sid = cursor + n + 1, *sst = sid + n_walks;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n, s);
    if (e != cudaSuccess) {
        scratch_free(buf, s);
        return cuda_fail(e, "cudaMemsetAsync(counts)");
    }
    const unsigned grid = blocks_for(n_walks, kThreads * 4);
    {
        ProfScope prof(kProfGroup, s);
        hist_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, counts, status);
        rc = scan_u32(counts, cursor, n, s);
        if (rc == BQ_OK) scatter_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, cursor, sid, sst);
        count_launches(2);
    }
    if (rc == BQ_OK) {
        // after the scatter cursor[v] is the end of bucket v; cursor[n] = valid walks
        switch (lanes_w) {
        case 1: launch_bouquet_w<RL, 1>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start,
                                        checked, agg, visits, paths, status, s); break;
        case 2: launch_bouquet_w<RL, 2>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start,
                                        checked, agg, visits, paths, status, s); break;
        case 8: launch_bouquet_w<RL, 8>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start,
                                        checked, agg, visits, paths, status, s); break;
        default: launch_bouquet_w<RL, 4>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start,
                                         checked, agg, visits, paths, status, s); break;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "walk_bouquet_kernel");
    }
    scratch_free(buf, s);
    return rc;
}

// The bouquet walk batch with every temporary buffer carved from a
// caller-provided scratch region (layout of launch_bouquet, scan workspace
// after it); used by the entry point that must not allocate.
template <typename RL>
int launch_bouquet_in(RL rl, const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                      uint32_t n_steps, const Sampler &smp, bool visit_start, bool checked, uint32_t *visits,
                      uint32_t *paths, uint32_t *status, int lanes_w, bool agg, char *scratch,
                      size_t scratch_bytes, size_t arrays_bytes, cudaStream_t s) {
    const size_t n = g.n;
    uint32_t *counts = (uint32_t *)scratch, *cursor = counts + n, *sid = cursor + n + 1, *sst = sid + n_walks;
    BQ_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n, s));
    const unsigned grid = blocks_for(n_walks, kThreads * 4);
    int rc;
    {
        ProfScope prof(kProfGroup, s);
        hist_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, counts, status);
        rc = scan_u32_ws(counts, cursor, n, scratch + arrays_bytes, scratch_bytes - arrays_bytes, s);
        if (rc == BQ_OK) scatter_starts_kernel<<<grid, kThreads, 0, s>>>(starts, n_walks, g.n, cursor, sid, sst);
        count_launches(2);
    }
    if (rc) return rc;
    switch (lanes_w) {
    case 1: launch_bouquet_w<RL, 1>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start, checked,
                                    agg, visits, paths, status, s); break;
    case 2: launch_bouquet_w<RL, 2>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start, checked,
                                    agg, visits, paths, status, s); break;
    case 8: launch_bouquet_w<RL, 8>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start, checked,
                                    agg, visits, paths, status, s); break;
    default: launch_bouquet_w<RL, 4>(rl, g, sid, sst, cursor + n, n_walks, n_steps, seed, smp, visit_start, checked,
                                     agg, visits, paths, status, s); break;
    }
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

size_t bouquet_arrays_bytes(uint32_t n, uint64_t n_walks) {
    return (sizeof(uint32_t) * (2 * (size_t)n + 1 + 2 * (size_t)n_walks) + 255) & ~(size_t)255;
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
    const uint64_t positions = (uint64_t)n_steps + (visit_start ? 1 : 0);
    const bool checked = positions > 0 && n_walks > 0xffffffffull / positions;
    const int lanes_w = tuning_walks_per_lane();
    const bool agg = tuning_aggregate_visits();
    const size_t arrays = bouquet_arrays_bytes(g.n, n_walks);
    if (g.compact())
        return launch_bouquet_in(RecCompact{g.rec8}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked,
                                 visits, paths, status, lanes_w, agg, (char *)scratch, scratch_bytes, arrays, s);
    return launch_bouquet_in(RecWide{g.rec16}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked, visits,
                             paths, status, lanes_w, agg, (char *)scratch, scratch_bytes, arrays, s);
}

int launch_walk_batch(const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                      uint32_t n_steps, uint32_t mode, const Sampler &smp, bool visit_start, uint32_t *visits,
                      uint32_t *paths, uint32_t *status, cudaStream_t s) {
    if (n_walks == 0) return BQ_OK;
    const uint64_t positions = (uint64_t)n_steps + (visit_start ? 1 : 0);
    // Below this bound a counter that starts at zero cannot wrap.
    const bool checked = positions > 0 && n_walks > 0xffffffffull / positions;
    const int lanes_w = tuning_walks_per_lane();
    const bool agg = tuning_aggregate_visits();
    if (mode == BQ_MODE_NAIVE) {
        if (g.compact())
            return launch_naive(RecCompact{g.rec8}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked,
                                visits, paths, status, s);
        return launch_naive(RecWide{g.rec16}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked,
                            visits, paths, status, s);
    }
    if (g.compact())
        return launch_bouquet(RecCompact{g.rec8}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked,
                              visits, paths, status, lanes_w, agg, s);
    return launch_bouquet(RecWide{g.rec16}, g, seed, starts, n_walks, n_steps, smp, visit_start, checked, visits,
                          paths, status, lanes_w, agg, s);
}

}  // namespace bq
