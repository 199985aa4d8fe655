// AESC kernels: the walk loop of TGT+ (Alg. 1) at zero push depth, turned
// into integer hit counters per query edge, and the final sum
// s(e) = g(u,v) + g(v,u) with g initialised to 1/d (Alg. 1).
//
// Work decomposition (GB300): a task is one bouquet of 32*W walks of one side
// of one edge, all starting at the same endpoint (Alg. 3 with B = 32*W).  A
// persistent grid of warps pulls tasks from a global counter; each lane
// advances W walks in lockstep, keeps its hit counts in registers, and the
// warp adds its two totals to the edge's counters with two atomics.
#include <math.h>

#include "edges.cuh"
#include "hash.cuh"
#include "internal.h"

namespace bq {
namespace {

constexpr int kThreads = 256;

struct QueryInfo {
    uint32_t u, v;    // normalised endpoints, u < v
    uint64_t edge;    // canonical id
    uint32_t du, dv;  // degrees
    uint32_t tau, nwalks;
    uint32_t valid;
    uint32_t depth;   // push depth (0 for the plain estimator)
};

// first index in [lo, hi) whose entry is >= key
__device__ __forceinline__ int64_t lower_bound_row(const uint32_t *__restrict__ nbrs, int64_t lo, int64_t hi,
                                                   uint32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (nbrs[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Canonical edge list: edge upper_before[u] + r is {u, r-th neighbour of u
// above u}.  One warp per vertex.
__global__ void canonical_edges_kernel(DeviceGraph g, uint32_t *__restrict__ uv) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = warp; u < g.n; u += nwarps) {
        const int64_t lo = g.offsets[u], hi = g.offsets[u + 1];
        const int64_t first = lower_bound_row(g.nbrs, lo, hi, (uint32_t)u + 1);
        const uint64_t id0 = g.upper_before[u];
        for (int64_t j = first + lane; j < hi; j += 32) {
            const uint64_t id = id0 + (uint64_t)(j - first);
            uv[2 * id] = (uint32_t)u;
            uv[2 * id + 1] = g.nbrs[j];
        }
    }
}

// push_max 0: the plain estimator.  push_max 1: push depth 1 where the push
// volume d(u) + d(v) is below the 2N walks it replaces (and tau >= 1); such
// an edge's walks are tau - 1 steps long, and none are run when that is 0.
__global__ void prepare_kernel(DeviceGraph g, const uint32_t *__restrict__ uv, uint64_t k,
                               const uint32_t *__restrict__ tau, const uint32_t *__restrict__ nwalks,
                               uint32_t bouquet, uint32_t push_max, QueryInfo *__restrict__ info,
                               uint32_t *__restrict__ tasks, uint32_t *__restrict__ depth_out,
                               double *__restrict__ sc, uint32_t *status) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        QueryInfo qi;
        const uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        qi.u = a < b ? a : b;
        qi.v = a < b ? b : a;
        qi.tau = tau[q];
        qi.nwalks = nwalks[q];
        qi.valid = 0;
        qi.edge = 0;
        qi.du = qi.dv = 0;
        qi.depth = 0;
        uint32_t status_bits = 0;
        if (a >= g.n || b >= g.n || a == b) {
            status_bits = kStatusNoEdge;
        } else {
            const int64_t lo = g.offsets[qi.u], hi = g.offsets[qi.u + 1];
            const int64_t pos = lower_bound_row(g.nbrs, lo, hi, qi.v);
            if (pos >= hi || g.nbrs[pos] != qi.v) {
                status_bits = kStatusNoEdge;
            } else {
                const int64_t first = lower_bound_row(g.nbrs, lo, hi, qi.u + 1);
                qi.edge = g.upper_before[qi.u] + (uint64_t)(pos - first);
                qi.du = (uint32_t)(hi - lo);
                qi.dv = (uint32_t)(g.offsets[qi.v + 1] - g.offsets[qi.v]);
                if (qi.tau == 0 || qi.nwalks == 0) status_bits = kStatusBadIndex;
                else if (2ull * qi.nwalks * qi.tau >= (1ull << 32)) status_bits = kStatusOverflow;
                else qi.valid = 1;
                if (qi.valid && push_max >= 1 && (uint64_t)qi.du + qi.dv < 2ull * qi.nwalks) qi.depth = 1;
            }
        }
        if (status_bits) atomicOr(status, status_bits);
        info[q] = qi;
        if (depth_out) depth_out[q] = qi.depth;
        tasks[q] = qi.valid && qi.tau > qi.depth ? 2u * ((qi.nwalks + bouquet - 1) / bouquet) : 0u;
        if (!qi.valid && sc) sc[q] = __longlong_as_double(0x7ff8000000000000ll);  // NaN
    }
}

// Persistent counting kernel.  Task t -> query q, side = local & 1, chunk =
// local >> 1; the chunk's walks are [chunk*32W, min(N, (chunk+1)*32W)).
// Independent sampler: lane l takes the W consecutive walks chunk*32W + l*W +
// j, so walk pairs (2i, 2i+1) share one Philox block.  Coupled sampler: slot
// j of lane l is walk chunk*32W + j*32 + l, so a coupling group of 32 fills
// one lockstep slot.
//
// HUB: the graph's hub table (the highest-degree vertex of each of hub_slots
// hash slots) is copied into shared memory with the hubs' vertex records, and
// a step that lands on a hub reads the record there instead of from L2/HBM.
// The grid is then 2 blocks of kHubAescThreads per SM (40 warps, the same as
// the plain kernel), each block with its own 12 B-per-slot copy of the table.
constexpr int kHubAescThreads = 640;

template <bool HUB>
constexpr int count_threads() {
    return HUB ? kHubAescThreads : kThreads;
}

// Resident blocks per SM the common shapes are compiled for: 40 warps
// (<= 48 registers) for both variants; the wider and coupled shapes keep
// their registers instead.
template <int W, bool COUPLED, bool HUB>
constexpr int count_min_blocks() {
    return (!COUPLED && W <= 4) ? (HUB ? 2 : 5) : 1;
}

template <typename EL, int W, bool COUPLED, bool HUB>
__global__ void __launch_bounds__(count_threads<HUB>(), count_min_blocks<W, COUPLED, HUB>())
aesc_count_kernel(EL el, const int64_t *__restrict__ offsets, const QueryInfo *__restrict__ info,
                  const uint64_t *__restrict__ begin, const uint32_t *__restrict__ bucket, uint64_t k,
                  uint64_t seed, Sampler smp, unsigned long long *__restrict__ next_task,
                  uint32_t *__restrict__ counts, const uint32_t *__restrict__ hub_tag, uint32_t hub_slots) {
    extern __shared__ __align__(16) unsigned char hub_smem[];
    uint2 *s_rec = reinterpret_cast<uint2 *>(hub_smem);
    const uint32_t slots = HUB ? hub_slots : 0u;
    uint32_t *s_tag = reinterpret_cast<uint32_t *>(s_rec + slots);
    if constexpr (HUB) {
        for (uint32_t i = threadIdx.x; i < slots; i += blockDim.x) {
            const uint32_t t = hub_tag[i];
            uint2 r = make_uint2(0u, 0u);
            if (t != kNoHub) {
                uint64_t o;
                uint32_t d;
                el.rec_of(t, o, d);
                r = make_uint2((uint32_t)o, d);
            }
            s_tag[i] = t;
            s_rec[i] = r;
        }
        __syncthreads();
    }
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t total = begin[k];
    const uint32_t shift = bucket_shift(total, k);
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const uint64_t q = task_edge(begin, bucket, k, total, shift, t);
        const QueryInfo qi = info[q];
        const uint64_t local = t - begin[q];
        const uint32_t side = (uint32_t)(local & 1);
        const uint64_t chunk = local >> 1;
        const uint64_t stream = 2 * qi.edge + side;
        const uint32_t start = side ? qi.v : qi.u;
        const uint64_t k0 = chunk * 32ull * W;

        uint64_t st[W], gs[W];
        uint32_t cur[W];
        bool act[W];
        if (!COUPLED && (W % 2 == 0)) {
#pragma unroll
            for (int j = 0; j < W; j += 2) {
                const uint64_t kk = k0 + (uint64_t)lane * W + j;
                walk_key_pair(seed, stream, kk >> 1, st[j], st[j + 1]);
                act[j] = kk < qi.nwalks;
                act[j + 1] = kk + 1 < qi.nwalks;
            }
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const uint64_t kk = COUPLED ? k0 + (uint64_t)j * 32 + lane : k0 + (uint64_t)lane * W + j;
                st[j] = walk_key(seed, stream, kk);
                if (COUPLED) gs[j] = walk_key(seed, stream | kGroupBit, kk / smp.width);
                act[j] = kk < qi.nwalks;
            }
        }
        uint64_t off0;
        uint32_t deg0;
        start_record(offsets, start, off0, deg0);
        uint64_t off[W];
        uint32_t deg[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            cur[j] = start;
            off[j] = off0;
            deg[j] = act[j] ? deg0 : 0u;  // inactive walks never move or hit
            if (!COUPLED) gs[j] = 0;
        }
        uint32_t hit_u = 0, hit_v = 0;
        for (uint32_t l = 1; l <= qi.tau; ++l) {
            const uint32_t weight = l < qi.tau ? 2u : 1u;
            if constexpr (HUB) {
                // the W walks' id loads, then their record loads, each issued
                // back to back so that a lane keeps W gathers in flight
                bool mv[W], hub[W];
                uint32_t slot[W];
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    st[j] += kGolden;
                    if (COUPLED) gs[j] += kGolden;
                    mv[j] = deg[j] != 0;
                    if (mv[j]) {
                        const uint32_t kk = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), deg[j]);
                        cur[j] = el.id(off[j] + kk);
                    }
                }
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    slot[j] = hub_slot(cur[j], slots);
                    hub[j] = mv[j] && s_tag[slot[j]] == cur[j];
                }
#pragma unroll
                for (int j = 0; j < W; ++j)
                    if (mv[j] && !hub[j]) el.rec_of(cur[j], off[j], deg[j]);
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    if (hub[j]) {
                        const uint2 r = s_rec[slot[j]];
                        off[j] = r.x;
                        deg[j] = r.y;
                    }
                    if (mv[j]) {
                        hit_u += cur[j] == qi.u ? weight : 0u;
                        hit_v += cur[j] == qi.v ? weight : 0u;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    st[j] += kGolden;
                    if (COUPLED) gs[j] += kGolden;
                    if (deg[j]) {
                        const uint32_t kk = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), deg[j]);
                        el.next(off[j] + kk, cur[j], off[j], deg[j]);
                        hit_u += cur[j] == qi.u ? weight : 0u;
                        hit_v += cur[j] == qi.v ? weight : 0u;
                    }
                }
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            hit_u += __shfl_down_sync(0xffffffffu, hit_u, d);
            hit_v += __shfl_down_sync(0xffffffffu, hit_v, d);
        }
        if (lane == 0) {
            if (hit_u) atomicAdd(counts + 4 * q + 2 * side + 0, hit_u);
            if (hit_v) atomicAdd(counts + 4 * q + 2 * side + 1, hit_v);
        }
    }
}

// The naive form of the same estimate (Alg. 2 per walk inside Alg. 1's walk
// loop): one walk per thread, walks in edge, side, walk order, on the plain
// CSR (a 4-byte neighbour id and the neighbour's vertex record per step), no
// bouquets, no task queue and no hub table.  Walk t of the flat order is
// walk w of side s of query q with begin[q] <= t < begin[q + 1], s = 1 when
// t - begin[q] >= N_q; it takes the same stream 2 e + s, walk index w and
// sampler as the bouquet kernel, so the counters are the same integers.  A
// walk with hits adds them to its side's two counters with its own atomics.
template <typename RL, bool COUPLED>
__global__ void __launch_bounds__(kThreads)
aesc_naive_kernel(RL rl, const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs,
                  const QueryInfo *__restrict__ info, const uint64_t *__restrict__ begin,
                  const uint32_t *__restrict__ bucket, uint64_t k, uint64_t seed, Sampler smp,
                  uint32_t *__restrict__ counts) {
    const uint64_t total = begin[k];
    const uint32_t shift = bucket_shift(total, k);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = task_edge(begin, bucket, k, total, shift, t);
        const QueryInfo qi = info[q];
        const uint64_t local = t - begin[q];
        const uint32_t side = local >= qi.nwalks ? 1u : 0u;
        const uint64_t w = local - (side ? qi.nwalks : 0u);
        const uint64_t stream = 2 * qi.edge + side;
        uint32_t cur = side ? qi.v : qi.u;
        uint64_t st = walk_key(seed, stream, w);
        uint64_t gs = COUPLED ? walk_key(seed, stream | kGroupBit, w / smp.width) : 0ull;
        uint64_t off;
        uint32_t deg;
        start_record(offsets, cur, off, deg);
        uint32_t hit_u = 0, hit_v = 0;
        for (uint32_t l = 1; l <= qi.tau; ++l) {
            st += kGolden;
            if (COUPLED) gs += kGolden;
            if (deg) {
                cur = nbrs[off + choose(sample_word<COUPLED>(st, gs, cur, smp.t), deg)];
                rl.load(cur, off, deg);
                const uint32_t weight = l < qi.tau ? 2u : 1u;
                hit_u += cur == qi.u ? weight : 0u;
                hit_v += cur == qi.v ? weight : 0u;
            }
        }
        if (hit_u) atomicAdd(counts + 4 * q + 2 * side + 0, hit_u);
        if (hit_v) atomicAdd(counts + 4 * q + 2 * side + 1, hit_v);
    }
}

struct NaiveRec8 {
    const uint2 *rec;
    __device__ __forceinline__ void load(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint2 r = __ldg(rec + v);
        off = r.x;
        deg = r.y;
    }
};

struct NaiveRec16 {
    const uint4 *rec;
    __device__ __forceinline__ void load(uint32_t v, uint64_t &off, uint32_t &deg) const {
        const uint4 r = __ldg(rec + v);
        off = ((uint64_t)r.y << 32) | r.x;
        deg = r.z;
    }
};

// Pilot sample of the scheduled plan: the first nwalks walks of each side,
// i.e. the estimator's own walks (same streams, walk indices and sampler),
// each scored by a = its weighted hits of u and b = its weighted hits of v.
// A lane keeps its two walks' scores apart; the warp adds the sums of a, b,
// a^2, b^2 and a b over its 64 walks to the side's five 64-bit moments
// moments[10q + 5 side + 0..4] with five atomics.
constexpr int kMomentW = 2;

template <typename EL, bool COUPLED>
__global__ void __launch_bounds__(kThreads)
aesc_moments_kernel(EL el, const int64_t *__restrict__ offsets, const QueryInfo *__restrict__ info,
                    const uint64_t *__restrict__ begin, const uint32_t *__restrict__ bucket, uint64_t k,
                    uint64_t seed, Sampler smp, unsigned long long *__restrict__ next_task,
                    unsigned long long *__restrict__ moments) {
    constexpr int W = kMomentW;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t total = begin[k];
    const uint32_t shift = bucket_shift(total, k);
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const uint64_t q = task_edge(begin, bucket, k, total, shift, t);
        const QueryInfo qi = info[q];
        const uint64_t local = t - begin[q];
        const uint32_t side = (uint32_t)(local & 1);
        const uint64_t k0 = (local >> 1) * 32ull * W;
        const uint64_t stream = 2 * qi.edge + side;
        const uint32_t start = side ? qi.v : qi.u;
        uint64_t st[W], gs[W];
        bool act[W];
        if constexpr (COUPLED) {
#pragma unroll
            for (int j = 0; j < W; ++j) {
                const uint64_t kk = k0 + (uint64_t)j * 32 + lane;
                st[j] = walk_key(seed, stream, kk);
                gs[j] = walk_key(seed, stream | kGroupBit, kk / smp.width);
                act[j] = kk < qi.nwalks;
            }
        } else {
            const uint64_t kk = k0 + (uint64_t)lane * W;
            walk_key_pair(seed, stream, kk >> 1, st[0], st[1]);
            gs[0] = gs[1] = 0;
            act[0] = kk < qi.nwalks;
            act[1] = kk + 1 < qi.nwalks;
        }
        uint64_t off0;
        uint32_t deg0;
        start_record(offsets, start, off0, deg0);
        uint64_t off[W];
        uint32_t cur[W], deg[W], ha[W], hb[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            cur[j] = start;
            off[j] = off0;
            deg[j] = act[j] ? deg0 : 0u;  // inactive walks never move or hit
            ha[j] = hb[j] = 0;
        }
        for (uint32_t l = 1; l <= qi.tau; ++l) {
            const uint32_t weight = l < qi.tau ? 2u : 1u;
#pragma unroll
            for (int j = 0; j < W; ++j) {
                st[j] += kGolden;
                if (COUPLED) gs[j] += kGolden;
                if (deg[j]) {
                    const uint32_t kk = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), deg[j]);
                    el.next(off[j] + kk, cur[j], off[j], deg[j]);
                    ha[j] += cur[j] == qi.u ? weight : 0u;
                    hb[j] += cur[j] == qi.v ? weight : 0u;
                }
            }
        }
        unsigned long long m[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
#pragma unroll
        for (int j = 0; j < W; ++j) {
            m[0] += ha[j];
            m[1] += hb[j];
            m[2] += (unsigned long long)ha[j] * ha[j];
            m[3] += (unsigned long long)hb[j] * hb[j];
            m[4] += (unsigned long long)ha[j] * hb[j];
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) m[i] += __shfl_down_sync(0xffffffffu, m[i], d);
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < 5; ++i)
                if (m[i]) atomicAdd(moments + 10 * q + 5 * side + i, m[i]);
        }
    }
}

// x - y of two unsigned integers as a double: the exact difference, rounded
// once.
__device__ __forceinline__ double signed_diff(uint64_t x, uint64_t y) {
    return x >= y ? __ull2double_rn(x - y) : -__ull2double_rn(y - x);
}

// Walk count of the pilot plan.  One sample of the estimator has the value
// Y = ((a(U) - a(V))/d_u + (b(V) - b(U))/d_v) / 2 with independent walks U
// from u and V from v, so Var Y = (Var_0 + Var_1) / 4 with, on side s,
// Var_s = Var a / d_u^2 + Var b / d_v^2 - 2 Cov(a, b) / (d_u d_v).  The
// unbiased sample moments come from the exact integer centred sums
// n0 S_aa - S_a^2, n0 S_bb - S_b^2, n0 S_ab - S_a S_b (exact in 64 bits while
// 2 n0 tau < 2^32); N = max(ceil(z^2 var / (eps/2)^2), n_min, 1).  Every FP64
// operation is rounded on its own (_rn intrinsics), in the documented order.
__global__ void pilot_nwalks_kernel(const QueryInfo *__restrict__ info, uint64_t k,
                                    const unsigned long long *__restrict__ moments, uint32_t n0, double eps,
                                    double z, uint32_t n_min, uint32_t *__restrict__ nwalks, uint32_t *status) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const QueryInfo qi = info[q];
        if (!qi.valid) {
            nwalks[q] = 0;
            continue;
        }
        const double du = (double)qi.du, dv = (double)qi.dv, n0d = (double)n0;
        double caa = 0.0, cbb = 0.0, cab = 0.0;
        for (int side = 0; side < 2; ++side) {
            const unsigned long long *m = moments + 10 * q + 5 * side;
            caa = __dadd_rn(caa, signed_diff((uint64_t)n0 * m[2], m[0] * m[0]));
            cbb = __dadd_rn(cbb, signed_diff((uint64_t)n0 * m[3], m[1] * m[1]));
            cab = __dadd_rn(cab, signed_diff((uint64_t)n0 * m[4], m[0] * m[1]));
        }
        const double num = __dsub_rn(__dadd_rn(__ddiv_rn(caa, __dmul_rn(du, du)), __ddiv_rn(cbb, __dmul_rn(dv, dv))),
                                     __ddiv_rn(__dmul_rn(2.0, cab), __dmul_rn(du, dv)));
        double var = __ddiv_rn(num, __dmul_rn(__dmul_rn(4.0, n0d), __dsub_rn(n0d, 1.0)));
        if (var < 0.0) var = 0.0;
        const double half = __dmul_rn(eps, 0.5);
        double nw = ceil(__ddiv_rn(__dmul_rn(__dmul_rn(z, z), var), __dmul_rn(half, half)));
        if (nw < (double)n_min) nw = (double)n_min;
        if (nw < 1.0) nw = 1.0;
        if (__dmul_rn(__dmul_rn(nw, 2.0), (double)qi.tau) >= 4294967296.0) {
            atomicOr(status, kStatusOverflow);
            nwalks[q] = 0;
        } else {
            nwalks[q] = (uint32_t)nw;
        }
    }
}

// s_e + ((C_uu - C_vu)/d_u + (C_vv - C_uv)/d_v) / (2N), every operation
// rounded to nearest on its own (explicit _rn intrinsics: no contraction).
__global__ void finalize_kernel(const QueryInfo *__restrict__ info, uint64_t k, const uint32_t *__restrict__ counts,
                                double *__restrict__ sc) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const QueryInfo qi = info[q];
        if (!qi.valid) continue;
        const double du = (double)qi.du, dv = (double)qi.dv;
        const double s = __dadd_rn(__ddiv_rn(1.0, du), __ddiv_rn(1.0, dv));
        const uint32_t c_uu = counts[4 * q + 0], c_uv = counts[4 * q + 1];
        const uint32_t c_vu = counts[4 * q + 2], c_vv = counts[4 * q + 3];
        const double x = (double)((int64_t)c_uu - (int64_t)c_vu);
        const double y = (double)((int64_t)c_vv - (int64_t)c_uv);
        const double mean = __ddiv_rn(__dadd_rn(__ddiv_rn(x, du), __ddiv_rn(y, dv)), __dmul_rn(2.0, (double)qi.nwalks));
        sc[q] = __dadd_rn(s, mean);
    }
}

// ------------------------------------------------------ AESC with a push phase

constexpr uint32_t kPushQ = 1u << 30;  // fixed-point scale of the pushed values

// Pushed value r_x(y) at depth 0 (Q [y == x]) or 1 (floor(Q / d_y) when y is
// a neighbour of x: a walk from y stands on x one step later with
// probability 1/d_y exactly then).  The row of x is searched in the plain
// CSR ids; every walk of a task searches the same two rows, which stay in L1.
__device__ __forceinline__ uint64_t pushed_value(const uint32_t *__restrict__ row, uint32_t d, uint32_t x,
                                                 uint32_t y, uint32_t dy, uint32_t depth) {
    if (depth == 0) return y == x ? (uint64_t)kPushQ : 0ull;
    return __ldg(row + last_le_row(row, d, y)) == y ? (uint64_t)(kPushQ / dy) : 0ull;  // d >= 1: x has an edge
}

// Per-warp shared-memory set of N(u) and N(v) for a depth-1 task with small
// rows: open addressing over kPushSetSlots slots (load <= 1/2), key = vertex
// id (kPushEmpty when free), flags bit 0 = neighbour of u, bit 1 = of v.
constexpr uint32_t kPushSetSlots = 128;
constexpr uint32_t kPushSetMaxRows = kPushSetSlots / 2;  // d(u) + d(v) admitted
constexpr uint32_t kPushEmpty = 0xffffffffu;

__device__ __forceinline__ uint32_t push_set_slot(uint32_t y) {
    return (y * 0x9E3779B1u) >> (32 - 7);  // 7 = log2(kPushSetSlots)
}

__device__ __forceinline__ void push_set_insert(uint32_t *keys, uint32_t *flags, uint32_t y, uint32_t bit) {
    uint32_t h = push_set_slot(y);
    for (uint32_t probe = 0; probe < kPushSetSlots; ++probe) {  // bounded: the set is at most half full
        const uint32_t prev = atomicCAS(keys + h, kPushEmpty, y);
        if (prev == kPushEmpty || prev == y) {
            atomicOr(flags + h, bit);
            return;
        }
        h = (h + 1) & (kPushSetSlots - 1);
    }
}

__device__ __forceinline__ uint32_t push_set_flags(const uint32_t *keys, const uint32_t *flags, uint32_t y) {
    uint32_t h = push_set_slot(y);
    for (uint32_t probe = 0; probe < kPushSetSlots; ++probe) {
        const uint32_t key = keys[h];
        if (key == y) return flags[h];
        if (key == kPushEmpty) return 0u;
        h = (h + 1) & (kPushSetSlots - 1);
    }
    return 0u;
}

// ---- push depths >= 2: pushed vectors r^j_x (r^0 = Q e_x, r^{j+1}(y) = sum
// over neighbours z of y of floor(r^j(z) / d_y)), built per query edge by one
// warp in two shared-memory hash tables, kept as sorted (vertex, value)
// arrays for the walks' lookups.
constexpr uint32_t kPushMaxDepth = 8;
constexpr uint32_t kPushSupportMax = kPushSupportCapMax;  // largest support cap per side and level
constexpr uint32_t kDeepSlots = 1024;      // hash slots per table (load <= 1/2 up to the cap)
constexpr int kDeepWarps = 8;              // warps per block of the build kernels
constexpr uint32_t kDeepEmpty = 0xffffffffu;

struct DeepInfo {
    uint64_t off;     // r_u's sorted table at tables[off], r_v's at tables[off + su]
    uint32_t su, sv;  // support sizes at the chosen depth
    int64_t xu, xv;   // sum over l <= depth of w_l (r^l_u(u) - r^l_u(v)), and for v
};

struct DeepTable {
    uint32_t keys[kDeepSlots];
    uint32_t vals[kDeepSlots];
    uint32_t count;  // distinct keys
    uint32_t over;   // count passed the cap (or the table filled)
};

struct DeepStats {
    uint64_t vol[2][kPushMaxDepth + 1];
    uint32_t supp[2][kPushMaxDepth + 1];
    uint32_t at_u[2][kPushMaxDepth + 1];
    uint32_t at_v[2][kPushMaxDepth + 1];
    uint32_t levels[2];
};

struct DeepWarp {
    DeepTable t[2];
    DeepStats st;
};

__device__ __forceinline__ uint32_t deep_hash(uint32_t y) { return (y * 0x9E3779B1u) >> 22; }  // 10 bits

__device__ void deep_clear(DeepTable *t, uint32_t lane) {
    for (uint32_t i = lane; i < kDeepSlots; i += 32) {
        t->keys[i] = kDeepEmpty;
        t->vals[i] = 0u;
    }
    if (lane == 0) {
        t->count = 0u;
        t->over = 0u;
    }
    __syncwarp();
}

__device__ void deep_add(DeepTable *t, uint32_t y, uint32_t c, uint32_t cap) {
    if (c == 0u) return;
    uint32_t h = deep_hash(y);
    for (uint32_t probe = 0; probe < kDeepSlots; ++probe) {
        const uint32_t prev = atomicCAS(t->keys + h, kDeepEmpty, y);
        if (prev == kDeepEmpty) {
            if (atomicAdd(&t->count, 1u) >= cap) t->over = 1u;
            atomicAdd(t->vals + h, c);
            return;
        }
        if (prev == y) {
            atomicAdd(t->vals + h, c);
            return;
        }
        h = (h + 1) & (kDeepSlots - 1);
    }
    t->over = 1u;
}

__device__ uint32_t deep_get(const DeepTable *t, uint32_t y) {
    uint32_t h = deep_hash(y);
    for (uint32_t probe = 0; probe < kDeepSlots; ++probe) {
        const uint32_t key = t->keys[h];
        if (key == y) return t->vals[h];
        if (key == kDeepEmpty) return 0u;
        h = (h + 1) & (kDeepSlots - 1);
    }
    return 0u;
}

// The volume of pushing `in`: the sum of the degrees of its support, the
// same in every lane.
__device__ uint64_t deep_volume(const int64_t *__restrict__ offsets, const DeepTable *in, uint32_t lane) {
    uint64_t vol = 0;
    for (uint32_t i = lane; i < kDeepSlots; i += 32) {
        const uint32_t z = in->keys[i];
        if (z != kDeepEmpty) vol += (uint64_t)(__ldg(offsets + z + 1) - __ldg(offsets + z));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) vol += __shfl_xor_sync(0xffffffffu, vol, d);
    return vol;
}

// out = one push of in.  Stops adding once out passed the cap (that level
// is then refused whatever else it would hold).
__device__ void deep_push(const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs,
                          const DeepTable *in, DeepTable *out, uint32_t cap, uint32_t lane) {
    deep_clear(out, lane);
    for (uint32_t i = lane; i < kDeepSlots; i += 32) {
        const uint32_t z = in->keys[i];
        if (z == kDeepEmpty) continue;
        const uint32_t r = in->vals[i];
        const int64_t lo = __ldg(offsets + z), hi = __ldg(offsets + z + 1);
        for (int64_t j = lo; j < hi; ++j) {
            if (*(volatile uint32_t *)&out->over) break;
            const uint32_t y = __ldg(nbrs + j);
            const uint32_t dy = (uint32_t)(__ldg(offsets + y + 1) - __ldg(offsets + y));
            deep_add(out, y, r / dy, cap);
        }
    }
    __syncwarp();
}

// Levels 0..jmax of source x into w->t (final level in t[result]); with
// limits, stops at a level whose volume reaches two_n (before pushing it) or
// after one whose support passes the cap (<= kPushSupportMax, which keeps
// the tables at most half full).  Records the per-level statistics of
// `side`.
__device__ uint32_t deep_levels(const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs, DeepWarp *w,
                                uint32_t side, uint32_t x, uint32_t u, uint32_t v, uint32_t jmax, bool limits,
                                uint64_t two_n, uint32_t cap, uint32_t lane) {
    deep_clear(&w->t[0], lane);
    if (lane == 0) deep_add(&w->t[0], x, kPushQ, cap);
    __syncwarp();
    if (lane == 0) {
        w->st.vol[side][0] = 0;
        w->st.supp[side][0] = 1;
        w->st.at_u[side][0] = x == u ? kPushQ : 0u;
        w->st.at_v[side][0] = x == v ? kPushQ : 0u;
        w->st.levels[side] = 0;
    }
    __syncwarp();
    uint32_t cur = 0;
    for (uint32_t j = 1; j <= jmax; ++j) {
        const uint64_t total = w->st.vol[side][j - 1] + deep_volume(offsets, &w->t[cur], lane);
        __syncwarp();
        if (limits && total >= two_n) {
            if (lane == 0) {
                w->st.vol[side][j] = total;
                w->st.supp[side][j] = 0;
                w->st.levels[side] = j;
            }
            __syncwarp();
            break;
        }
        deep_push(offsets, nbrs, &w->t[cur], &w->t[cur ^ 1], cap, lane);
        cur ^= 1;
        const DeepTable *t = &w->t[cur];
        const uint32_t supp = t->count, over = t->over;
        const uint32_t au = deep_get(t, u), av = deep_get(t, v);
        __syncwarp();
        if (lane == 0) {
            w->st.vol[side][j] = total;
            w->st.supp[side][j] = supp;
            w->st.at_u[side][j] = au;
            w->st.at_v[side][j] = av;
            w->st.levels[side] = j;
        }
        __syncwarp();
        if (limits && (over || supp > cap)) break;
    }
    return cur;
}

// Pass 1: for each query at depth 1 with push_max >= 2 and tau >= 2, the
// deepest level every rule admits (volumes of both sides below 2N, supports
// within the cap); deeper queries get their depth, X terms, support sizes
// and walk tasks.
__global__ void __launch_bounds__(kDeepWarps * 32)
deep_plan_kernel(const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs, QueryInfo *__restrict__ info,
                 uint64_t k, uint32_t push_max, uint32_t cap, uint32_t bouquet, DeepInfo *__restrict__ deep,
                 uint32_t *__restrict__ sizes, uint32_t *__restrict__ tasks) {
    extern __shared__ __align__(16) unsigned char deep_smem[];
    DeepWarp *w = reinterpret_cast<DeepWarp *>(deep_smem) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = warp; q < k; q += nwarps) {
        const QueryInfo qi = info[q];
        uint32_t jmax = push_max < qi.tau ? push_max : qi.tau;
        if (jmax > kPushMaxDepth) jmax = kPushMaxDepth;
        if (lane == 0) sizes[q] = 0u;
        if (!qi.valid || qi.depth != 1 || jmax < 2) continue;
        const uint64_t two_n = 2ull * qi.nwalks;
        // level 2 needs both rows within the cap and vol_2(x) = d_x + the sum
        // of the degrees of N(x) below 2N in total: most edges stop here
        if (qi.du > cap || qi.dv > cap) continue;
        uint64_t vol2 = 0;
        const int64_t lu = __ldg(offsets + qi.u), lv = __ldg(offsets + qi.v);
        for (uint32_t i = lane; i < qi.du; i += 32) {
            const uint32_t z = __ldg(nbrs + lu + i);
            vol2 += (uint64_t)(__ldg(offsets + z + 1) - __ldg(offsets + z));
        }
        for (uint32_t i = lane; i < qi.dv; i += 32) {
            const uint32_t z = __ldg(nbrs + lv + i);
            vol2 += (uint64_t)(__ldg(offsets + z + 1) - __ldg(offsets + z));
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) vol2 += __shfl_xor_sync(0xffffffffu, vol2, d);
        if ((uint64_t)qi.du + qi.dv + vol2 >= two_n) continue;
        deep_levels(offsets, nbrs, w, 0, qi.u, qi.u, qi.v, jmax, true, two_n, cap, lane);
        deep_levels(offsets, nbrs, w, 1, qi.v, qi.u, qi.v, jmax, true, two_n, cap, lane);
        if (lane == 0) {
            const DeepStats &st = w->st;
            const uint32_t top = st.levels[0] < st.levels[1] ? st.levels[0] : st.levels[1];
            uint32_t dep = 0;
            for (uint32_t j = 1; j <= top; ++j) {
                if (st.vol[0][j] + st.vol[1][j] >= two_n) break;
                if (j >= 2 && (st.supp[0][j] > cap || st.supp[1][j] > cap)) break;
                dep = j;
            }
            if (dep >= 2) {
                int64_t xu = 0, xv = 0;
                for (uint32_t l = 0; l <= dep; ++l) {
                    const int64_t wl = l < qi.tau ? 2 : 1;
                    xu += wl * ((int64_t)st.at_u[0][l] - (int64_t)st.at_v[0][l]);
                    xv += wl * ((int64_t)st.at_v[1][l] - (int64_t)st.at_u[1][l]);
                }
                DeepInfo di;
                di.off = 0;
                di.su = st.supp[0][dep];
                di.sv = st.supp[1][dep];
                di.xu = xu;
                di.xv = xv;
                deep[q] = di;
                sizes[q] = di.su + di.sv;
                info[q].depth = dep;
                tasks[q] = qi.tau > dep ? 2u * ((qi.nwalks + bouquet - 1) / bouquet) : 0u;
            }
        }
        __syncwarp();
    }
}

// Pass 2: the pushed vectors of each deeper query at its depth, as sorted
// (vertex << 32 | value) arrays at tables[toff[q]] (r_u, then r_v).
__global__ void __launch_bounds__(kDeepWarps * 32)
deep_tables_kernel(const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs,
                   const QueryInfo *__restrict__ info, uint64_t k, const uint64_t *__restrict__ toff,
                   DeepInfo *__restrict__ deep, unsigned long long *__restrict__ tables) {
    extern __shared__ __align__(16) unsigned char deep_smem[];
    DeepWarp *w = reinterpret_cast<DeepWarp *>(deep_smem) + (threadIdx.x >> 5);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t q = warp; q < k; q += nwarps) {
        const QueryInfo qi = info[q];
        if (!qi.valid || qi.depth < 2) continue;
        const uint64_t base = toff[q];
        if (lane == 0) deep[q].off = base;
        uint64_t at = base;
        for (uint32_t side = 0; side < 2; ++side) {
            // every level up to the depth passed the planner's cap in pass 1
            const uint32_t fin = deep_levels(offsets, nbrs, w, side, side ? qi.v : qi.u, qi.u, qi.v, qi.depth,
                                             false, 0, kPushSupportMax, lane);
            const DeepTable *t = &w->t[fin];
            // compact into the other table's memory, pad to a power of two, sort
            unsigned long long *arr = reinterpret_cast<unsigned long long *>(&w->t[fin ^ 1]);
            uint32_t n_out = 0;
            for (uint32_t base_i = 0; base_i < kDeepSlots; base_i += 32) {
                const uint32_t i = base_i + lane;
                const uint32_t key = t->keys[i];
                const bool has = key != kDeepEmpty;
                const uint32_t mask = __ballot_sync(0xffffffffu, has);
                if (has) {
                    const uint32_t pos = n_out + __popc(mask & ((1u << lane) - 1u));
                    arr[pos] = ((unsigned long long)key << 32) | t->vals[i];
                }
                n_out += __popc(mask);
            }
            uint32_t p2 = 1;
            while (p2 < n_out) p2 <<= 1;
            for (uint32_t i = n_out + lane; i < p2; i += 32) arr[i] = ~0ull;
            __syncwarp();
            for (uint32_t kk = 2; kk <= p2; kk <<= 1) {
                for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
                    for (uint32_t i = lane; i < p2; i += 32) {
                        const uint32_t ixj = i ^ jj;
                        if (ixj > i) {
                            const unsigned long long a = arr[i], b = arr[ixj];
                            const bool up = (i & kk) == 0;
                            if ((a > b) == up) {
                                arr[i] = b;
                                arr[ixj] = a;
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            for (uint32_t i = lane; i < n_out; i += 32) tables[at + i] = arr[i];
            at += n_out;
            __syncwarp();
        }
    }
}

// r_x(y) from a sorted (vertex << 32 | value) array of `size` entries: the
// last entry whose vertex is <= y, found in a trip count that depends on the
// size alone (all lanes of a task search the same table).
__device__ __forceinline__ uint64_t deep_value(const unsigned long long *__restrict__ tab, uint32_t size,
                                               uint32_t y) {
    if (size == 0) return 0ull;
    uint32_t base = 0;
    while (size > 1) {
        const uint32_t half = size >> 1;
        if ((uint32_t)(__ldg(tab + base + half) >> 32) <= y) base += half;
        size -= half;
    }
    const unsigned long long e = __ldg(tab + base);
    return (uint32_t)(e >> 32) == y ? (e & 0xffffffffull) : 0ull;
}

// Persistent counting kernel of the push estimator: the tasks, streams and
// walk indices of aesc_count_kernel (independent sampler), walks of tau -
// depth steps; at step l a walk adds w r_u(cur) and w r_v(cur), w = 2 if
// l + depth < tau else 1, to 64-bit fixed-point accumulators
// acc[4q + 2 side + {0, 1}] (A_uu, A_uv from u; A_vu, A_vv from v).
// Resident blocks per SM the push kernel is compiled for.  It waits on
// dependent loads, so occupancy pays: 6 blocks (40 registers) at 2 walks per
// lane and 5 (48) at 4 were measured 16 % and 4-9 % faster than 4 blocks, and 8
// blocks (32 registers, spilling) slower than 6.
template <int W>
constexpr int push_min_blocks() {
    return W <= 2 ? 6 : (W <= 4 ? 5 : 1);
}

template <typename EL, int W>
__global__ void __launch_bounds__(kThreads, push_min_blocks<W>())
aesc_push_kernel(EL el, const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs,
                 const QueryInfo *__restrict__ info, const uint64_t *__restrict__ begin,
                 const uint32_t *__restrict__ bucket, uint64_t k, uint64_t seed,
                 unsigned long long *__restrict__ next_task, unsigned long long *__restrict__ acc,
                 const DeepInfo *__restrict__ deep, const unsigned long long *__restrict__ tables) {
    __shared__ uint32_t s_keys[kThreads / 32][kPushSetSlots];
    __shared__ uint32_t s_flags[kThreads / 32][kPushSetSlots];
    const uint32_t lane = threadIdx.x & 31;
    uint32_t *keys = s_keys[threadIdx.x >> 5];
    uint32_t *flags = s_flags[threadIdx.x >> 5];
    const uint64_t total = begin[k];
    const uint32_t shift = bucket_shift(total, k);
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const uint64_t q = task_edge(begin, bucket, k, total, shift, t);
        const QueryInfo qi = info[q];
        const uint64_t local = t - begin[q];
        const uint32_t side = (uint32_t)(local & 1);
        const uint64_t stream = 2 * qi.edge + side;
        const uint32_t start = side ? qi.v : qi.u;
        const uint64_t k0 = (local >> 1) * 32ull * W;
        const int64_t lo_u = __ldg(offsets + qi.u), lo_v = __ldg(offsets + qi.v);
        const uint32_t *__restrict__ row_u = nbrs + lo_u;
        const uint32_t *__restrict__ row_v = nbrs + lo_v;
        // small rows at depth 1: the warp hashes N(u) and N(v) into its set
        const bool use_set = qi.depth == 1 && (uint64_t)qi.du + qi.dv <= kPushSetMaxRows;
        // depths >= 2: the edge's sorted pushed vectors
        const unsigned long long *tab_u = nullptr, *tab_v = nullptr;
        uint32_t size_u = 0, size_v = 0;
        if (qi.depth >= 2) {
            const DeepInfo di = deep[q];
            tab_u = tables + di.off;
            tab_v = tab_u + di.su;
            size_u = di.su;
            size_v = di.sv;
        }
        if (use_set) {
            for (uint32_t i = lane; i < kPushSetSlots; i += 32) {
                keys[i] = kPushEmpty;
                flags[i] = 0u;
            }
            __syncwarp();
            for (uint32_t i = lane; i < qi.du; i += 32) push_set_insert(keys, flags, __ldg(row_u + i), 1u);
            for (uint32_t i = lane; i < qi.dv; i += 32) push_set_insert(keys, flags, __ldg(row_v + i), 2u);
            __syncwarp();
        }

        uint64_t st[W];
        uint32_t cur[W], deg[W];
        uint64_t off[W];
        bool act[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t kk = k0 + (uint64_t)lane * W + j;
            st[j] = walk_key(seed, stream, kk);
            act[j] = kk < qi.nwalks;
        }
        uint64_t off0;
        uint32_t deg0;
        start_record(offsets, start, off0, deg0);
#pragma unroll
        for (int j = 0; j < W; ++j) {
            cur[j] = start;
            off[j] = off0;
            deg[j] = act[j] ? deg0 : 0u;
        }
        uint64_t a_u = 0, a_v = 0;
        const uint32_t steps = qi.tau - qi.depth;
        // the walk loop with one lookup of the pushed values, chosen per task
        auto walk = [&](auto lookup) {
            for (uint32_t l = 1; l <= steps; ++l) {
                const uint64_t weight = l + qi.depth < qi.tau ? 2ull : 1ull;
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    st[j] += kGolden;
                    if (deg[j]) {
                        const uint32_t kk = choose(sample_word<false>(st[j], 0ull, cur[j], 0u), deg[j]);
                        el.next(off[j] + kk, cur[j], off[j], deg[j]);
                        lookup(cur[j], deg[j], weight);
                    }
                }
            }
        };
        if (qi.depth >= 2) {
            walk([&](uint32_t y, uint32_t, uint64_t weight) {
                a_u += weight * deep_value(tab_u, size_u, y);
                a_v += weight * deep_value(tab_v, size_v, y);
            });
        } else if (use_set) {
            walk([&](uint32_t y, uint32_t dy, uint64_t weight) {
                const uint32_t f = push_set_flags(keys, flags, y);
                if (f) {
                    const uint64_t r = (uint64_t)(kPushQ / dy);
                    if (f & 1u) a_u += weight * r;
                    if (f & 2u) a_v += weight * r;
                }
            });
        } else {
            walk([&](uint32_t y, uint32_t dy, uint64_t weight) {
                a_u += weight * pushed_value(row_u, qi.du, qi.u, y, dy, qi.depth);
                a_v += weight * pushed_value(row_v, qi.dv, qi.v, y, dy, qi.depth);
            });
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            a_u += __shfl_down_sync(0xffffffffu, a_u, d);
            a_v += __shfl_down_sync(0xffffffffu, a_v, d);
        }
        if (lane == 0) {
            if (a_u) atomicAdd(acc + 4 * q + 2 * side + 0, (unsigned long long)a_u);
            if (a_v) atomicAdd(acc + 4 * q + 2 * side + 1, (unsigned long long)a_v);
        }
    }
}

// g(u, v) = (X_u + (A_uu - A_vu) / N) / (2 Q d_u) with X_u = 2Q, less
// w_1 floor(Q / d_v) at depth 1 (w_1 = 2 if tau > 1 else 1), and at depths
// >= 2 the sum over l <= depth of w_l (r^l_u(u) - r^l_u(v)) from the build;
// SC = g(u, v) + g(v, u); every operation rounded to nearest on its own, in
// this order.
__global__ void finalize_push_kernel(const QueryInfo *__restrict__ info, uint64_t k,
                                     const unsigned long long *__restrict__ acc, const DeepInfo *__restrict__ deep,
                                     double *__restrict__ sc) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const QueryInfo qi = info[q];
        if (!qi.valid) continue;
        int64_t xu = 2 * (int64_t)kPushQ, xv = 2 * (int64_t)kPushQ;
        if (qi.depth == 1) {
            const int64_t w1 = qi.tau > 1 ? 2 : 1;
            xu -= w1 * (int64_t)(kPushQ / qi.dv);
            xv -= w1 * (int64_t)(kPushQ / qi.du);
        } else if (qi.depth >= 2) {
            xu = deep[q].xu;
            xv = deep[q].xv;
        }
        const double du = (double)qi.du, dv = (double)qi.dv, nw = (double)qi.nwalks;
        const double yu = (double)(int64_t)(acc[4 * q + 0] - acc[4 * q + 2]);
        const double yv = (double)(int64_t)(acc[4 * q + 3] - acc[4 * q + 1]);
        const double gu = __ddiv_rn(__dadd_rn((double)xu, __ddiv_rn(yu, nw)), __dmul_rn(2.0 * (double)kPushQ, du));
        const double gv = __ddiv_rn(__dadd_rn((double)xv, __ddiv_rn(yv, nw)), __dmul_rn(2.0 * (double)kPushQ, dv));
        sc[q] = __dadd_rn(gu, gv);
    }
}

// The push depth of every query, once pass 1 of the deeper pushes has run.
__global__ void push_depth_out_kernel(const QueryInfo *__restrict__ info, uint64_t k, uint32_t *__restrict__ depth) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x)
        depth[q] = info[q].depth;
}

unsigned blocks_for(uint64_t items, uint64_t per_block) {
    uint64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 0x7fffffffull) b = 0x7fffffffull;
    return (unsigned)b;
}

// The hub variant when the graph has a hub table and a split layout (a
// separate vertex-record load per step) and the table fits; else the plain
// kernel.
template <typename EL, int W, bool COUPLED>
int launch_count(EL el, const DeviceGraph &g, const QueryInfo *info, const uint64_t *begin, uint64_t k,
                 uint64_t seed, const Sampler &smp, unsigned long long *next_task, uint32_t *counts,
                 cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the bucket table follows begin[k + 1] in the scratch buffer
    const uint32_t *bucket = reinterpret_cast<const uint32_t *>(begin + k + 1);
    if constexpr (EL::kSplit) {
        if (g.hub_tag && g.rec8 && tuning_aesc_hub()) {
            const size_t smem = (size_t)12 * g.hub_slots;
            auto kernel = aesc_count_kernel<EL, W, COUPLED, true>;
            if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kHubAescThreads, smem) == cudaSuccess &&
                per_sm >= 1) {
                kernel<<<sms * per_sm, kHubAescThreads, smem, s>>>(el, g.offsets, info, begin, bucket, k, seed, smp,
                                                                  next_task, counts, g.hub_tag, g.hub_slots);
                BQ_CUDA(cudaGetLastError());
                return BQ_OK;
            }
            cudaGetLastError();
        }
    }
    auto kernel = aesc_count_kernel<EL, W, COUPLED, false>;
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    kernel<<<sms * per_sm, kThreads, 0, s>>>(el, g.offsets, info, begin, bucket, k, seed, smp, next_task, counts,
                                             nullptr, 0);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

template <typename EL>
int launch_count_w(EL el, const DeviceGraph &g, const QueryInfo *info, const uint64_t *begin, uint64_t k,
                   uint64_t seed, const Sampler &smp, unsigned long long *next_task, uint32_t *counts,
                   int w, cudaStream_t s) {
    const bool coupled = smp.kind == 1;
    switch (w) {
    case 2:
        return coupled ? launch_count<EL, 2, true>(el, g, info, begin, k, seed, smp, next_task, counts, s)
                       : launch_count<EL, 2, false>(el, g, info, begin, k, seed, smp, next_task, counts, s);
    case 8:
        return coupled ? launch_count<EL, 8, true>(el, g, info, begin, k, seed, smp, next_task, counts, s)
                       : launch_count<EL, 8, false>(el, g, info, begin, k, seed, smp, next_task, counts, s);
    default:
        return coupled ? launch_count<EL, 4, true>(el, g, info, begin, k, seed, smp, next_task, counts, s)
                       : launch_count<EL, 4, false>(el, g, info, begin, k, seed, smp, next_task, counts, s);
    }
}

}  // namespace

int launch_canonical_edges(const DeviceGraph &g, uint32_t *uv, cudaStream_t s) {
    if (g.n == 0) return BQ_OK;
    count_launches(1);
    canonical_edges_kernel<<<blocks_for((uint64_t)g.n * 32, kThreads), kThreads, 0, s>>>(g, uv);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

// One walk per thread over the flat walk order (grid-stride, a grid of SMs x
// resident blocks).
template <typename RL>
int launch_naive_count(RL rl, const DeviceGraph &g, const QueryInfo *info, const uint64_t *begin, uint64_t k,
                       uint64_t seed, const Sampler &smp, uint32_t *counts, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t *bucket = reinterpret_cast<const uint32_t *>(begin + k + 1);
    if (smp.kind == 1) {
        auto kernel = aesc_naive_kernel<RL, true>;
        BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
        kernel<<<sms * (per_sm < 1 ? 1 : per_sm), kThreads, 0, s>>>(rl, g.offsets, g.nbrs, info, begin, bucket, k,
                                                                    seed, smp, counts);
    } else {
        auto kernel = aesc_naive_kernel<RL, false>;
        BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
        kernel<<<sms * (per_sm < 1 ? 1 : per_sm), kThreads, 0, s>>>(rl, g.offsets, g.nbrs, info, begin, bucket, k,
                                                                    seed, smp, counts);
    }
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

int launch_aesc(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k, const uint32_t *tau,
                const uint32_t *nwalks, const Sampler &smp, bool naive, uint32_t *counts, double *sc,
                uint32_t *status, cudaStream_t s) {
    if (k == 0) return BQ_OK;
    int w = tuning_aesc_walks_per_lane();
    if (w != 2 && w != 4 && w != 8) w = 4;
    // the naive kernel's work items are single walks: 2 N per edge
    const uint32_t bouquet = naive ? 1u : 32u * (uint32_t)w;
    if (k >= kMaxBucketEdges) return fail(BQ_EINVAL, "k = %llu edges in one estimate", (unsigned long long)k);
    // scratch: info[k] | begin[k + 1] bucket[k + 1] | tasks[k] | next_task |
    // (edges[2k] if all-edges)
    const size_t info_bytes = sizeof(QueryInfo) * k;
    const size_t begin_bytes = sizeof(uint64_t) * (k + 1) + ((sizeof(uint32_t) * bucket_count(k) + 7) & ~(size_t)7);
    const size_t task_bytes = sizeof(uint32_t) * ((k + 1) & ~1ull);
    const size_t edge_bytes = edges_uv ? 0 : sizeof(uint32_t) * 2 * k;
    const size_t bytes = info_bytes + begin_bytes + task_bytes + 16 + edge_bytes;
    char *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, bytes, s);
    if (rc) return rc;
    QueryInfo *info = (QueryInfo *)buf;
    uint64_t *begin = (uint64_t *)(buf + info_bytes);
    uint32_t *tasks = (uint32_t *)(buf + info_bytes + begin_bytes);
    unsigned long long *next_task = (unsigned long long *)(buf + info_bytes + begin_bytes + task_bytes);
    uint32_t *all_uv = (uint32_t *)(buf + info_bytes + begin_bytes + task_bytes + 16);
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * 4 * k, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next_task, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        scratch_free(buf, s);
        return cuda_fail(e, "aesc setup");
    }
    const uint32_t *uv = edges_uv;
    {
        ProfScope prof(kProfAescAux, s);
        if (!uv) {
            count_launches(1);
            canonical_edges_kernel<<<blocks_for((uint64_t)g.n * 32, kThreads), kThreads, 0, s>>>(g, all_uv);
            uv = all_uv;
        }
        count_launches(1);
        prepare_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(g, uv, k, tau, nwalks, bouquet, 0u, info, tasks,
                                                                    nullptr, sc, status);
        rc = scan_u32_to_u64(tasks, begin, k, s);
        if (rc == BQ_OK) {
            count_launches(1);
            build_bucket_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(
                begin, k, reinterpret_cast<uint32_t *>(begin + k + 1));
        }
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        if (naive)
            rc = g.compact() ? launch_naive_count(NaiveRec8{g.rec8}, g, info, begin, k, seed, smp, counts, s)
                             : launch_naive_count(NaiveRec16{g.rec16}, g, info, begin, k, seed, smp, counts, s);
        else
            rc = with_edges(g, [&](auto el) {
                return launch_count_w(el, g, info, begin, k, seed, smp, next_task, counts, w, s);
            });
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        finalize_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(info, k, counts, sc);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "finalize_kernel");
    }
    scratch_free(buf, s);
    return rc;
}

}  // namespace bq

namespace bq {
namespace {

template <typename EL, int W>
int launch_push_count(EL el, const DeviceGraph &g, const QueryInfo *info, const uint64_t *begin, uint64_t k,
                      uint64_t seed, unsigned long long *next_task, unsigned long long *acc, const DeepInfo *deep,
                      const unsigned long long *tables, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kernel = aesc_push_kernel<EL, W>;
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const uint32_t *bucket = reinterpret_cast<const uint32_t *>(begin + k + 1);
    kernel<<<sms * per_sm, kThreads, 0, s>>>(el, g.offsets, g.nbrs, info, begin, bucket, k, seed, next_task, acc,
                                             deep, tables);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

// Depths >= 2: plan (pass 1), size and allocate the tables (one wait on s),
// build them (pass 2).  *tables_out is released by the caller.
int build_deep(const DeviceGraph &g, QueryInfo *info, uint64_t k, uint32_t push_max, uint32_t cap,
               uint32_t bouquet, DeepInfo *deep, uint32_t *sizes, uint64_t *toff, uint32_t *tasks,
               unsigned long long **tables_out, cudaStream_t s) {
    *tables_out = nullptr;
    const size_t smem = sizeof(DeepWarp) * kDeepWarps;
    BQ_CUDA(cudaFuncSetAttribute(deep_plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BQ_CUDA(cudaFuncSetAttribute(deep_tables_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned grid = blocks_for(k, kDeepWarps) < (unsigned)sms ? blocks_for(k, kDeepWarps) : (unsigned)sms;
    count_launches(1);
    deep_plan_kernel<<<grid, kDeepWarps * 32, smem, s>>>(g.offsets, g.nbrs, info, k, push_max, cap, bouquet, deep,
                                                         sizes, tasks);
    BQ_CUDA(cudaGetLastError());
    int rc = scan_u32_to_u64(sizes, toff, k, s);
    if (rc) return rc;
    uint64_t total = 0;
    BQ_CUDA(cudaMemcpyAsync(&total, toff + k, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
    BQ_CUDA(cudaStreamSynchronize(s));
    if (total == 0) return BQ_OK;
    unsigned long long *tables = nullptr;
    rc = scratch_alloc((void **)&tables, sizeof(unsigned long long) * total, s);
    if (rc) return rc;
    count_launches(1);
    deep_tables_kernel<<<grid, kDeepWarps * 32, smem, s>>>(g.offsets, g.nbrs, info, k, toff, deep, tables);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        scratch_free(tables, s);
        return cuda_fail(e, "deep_tables_kernel");
    }
    *tables_out = tables;
    return BQ_OK;
}

}  // namespace

int launch_aesc_push(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k, const uint32_t *tau,
                     const uint32_t *nwalks, uint32_t push_max, uint32_t support_cap, uint32_t *depth_out,
                     uint64_t *acc, double *sc, uint32_t *status, cudaStream_t s) {
    if (k == 0) return BQ_OK;
    int w = tuning_push_walks_per_lane();
    if (w != 2 && w != 4 && w != 8) w = 2;
    const uint32_t bouquet = 32u * (uint32_t)w;
    if (k >= kMaxBucketEdges) return fail(BQ_EINVAL, "k = %llu edges in one estimate", (unsigned long long)k);
    const bool deep_on = push_max >= 2;
    // scratch: info[k] | begin[k + 1] bucket[k + 1] | tasks[k] | next_task |
    // (edges[2k] if all-edges) | (deep[k] sizes[k] toff[k + 1] if push_max >= 2)
    const size_t info_bytes = sizeof(QueryInfo) * k;
    const size_t begin_bytes = sizeof(uint64_t) * (k + 1) + ((sizeof(uint32_t) * bucket_count(k) + 7) & ~(size_t)7);
    const size_t task_bytes = sizeof(uint32_t) * ((k + 1) & ~1ull);
    const size_t edge_bytes = edges_uv ? 0 : sizeof(uint32_t) * 2 * k;
    const size_t deep_bytes = deep_on ? sizeof(DeepInfo) * k : 0;
    const size_t size_bytes = deep_on ? sizeof(uint32_t) * ((k + 1) & ~1ull) : 0;
    const size_t toff_bytes = deep_on ? sizeof(uint64_t) * (k + 1) : 0;
    const size_t head = info_bytes + begin_bytes + task_bytes + 16 + ((edge_bytes + 15) & ~(size_t)15);
    const size_t bytes = head + deep_bytes + size_bytes + toff_bytes;
    char *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, bytes, s);
    if (rc) return rc;
    QueryInfo *info = (QueryInfo *)buf;
    uint64_t *begin = (uint64_t *)(buf + info_bytes);
    uint32_t *tasks = (uint32_t *)(buf + info_bytes + begin_bytes);
    unsigned long long *next_task = (unsigned long long *)(buf + info_bytes + begin_bytes + task_bytes);
    uint32_t *all_uv = (uint32_t *)(buf + info_bytes + begin_bytes + task_bytes + 16);
    DeepInfo *deep = deep_on ? (DeepInfo *)(buf + head) : nullptr;
    uint32_t *sizes = deep_on ? (uint32_t *)(buf + head + deep_bytes) : nullptr;
    uint64_t *toff = deep_on ? (uint64_t *)(buf + head + deep_bytes + size_bytes) : nullptr;
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(acc);
    unsigned long long *tables = nullptr;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(uint64_t) * 4 * k, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next_task, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        scratch_free(buf, s);
        return cuda_fail(e, "aesc push setup");
    }
    const uint32_t *uv = edges_uv;
    {
        ProfScope prof(kProfAescAux, s);
        if (!uv) {
            count_launches(1);
            canonical_edges_kernel<<<blocks_for((uint64_t)g.n * 32, kThreads), kThreads, 0, s>>>(g, all_uv);
            uv = all_uv;
        }
        count_launches(1);
        prepare_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(g, uv, k, tau, nwalks, bouquet, push_max, info,
                                                                    tasks, nullptr, sc, status);
        if (deep_on)
            rc = build_deep(g, info, k, push_max, support_cap, bouquet, deep, sizes, toff, tasks, &tables, s);
        if (rc == BQ_OK) rc = scan_u32_to_u64(tasks, begin, k, s);
        if (rc == BQ_OK) {
            count_launches(1);
            build_bucket_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(
                begin, k, reinterpret_cast<uint32_t *>(begin + k + 1));
        }
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        rc = with_edges(g, [&](auto el) {
            using EL = decltype(el);
            if (w == 2) return launch_push_count<EL, 2>(el, g, info, begin, k, seed, next_task, acc64, deep, tables, s);
            if (w == 8) return launch_push_count<EL, 8>(el, g, info, begin, k, seed, next_task, acc64, deep, tables, s);
            return launch_push_count<EL, 4>(el, g, info, begin, k, seed, next_task, acc64, deep, tables, s);
        });
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAescAux, s);
        count_launches(depth_out ? 2 : 1);
        finalize_push_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(info, k, acc64, deep, sc);
        if (depth_out) push_depth_out_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(info, k, depth_out);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "finalize_push_kernel");
    }
    if (tables) scratch_free(tables, s);
    scratch_free(buf, s);
    return rc;
}

}  // namespace bq

namespace bq {
namespace {

template <typename EL, bool COUPLED>
int launch_moments(EL el, const DeviceGraph &g, const QueryInfo *info, const uint64_t *begin, uint64_t k,
                   uint64_t seed, const Sampler &smp, unsigned long long *next_task, unsigned long long *moments,
                   cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kernel = aesc_moments_kernel<EL, COUPLED>;
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const uint32_t *bucket = reinterpret_cast<const uint32_t *>(begin + k + 1);
    kernel<<<sms * per_sm, kThreads, 0, s>>>(el, g.offsets, info, begin, bucket, k, seed, smp, next_task, moments);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

}  // namespace

int launch_aesc_moments(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k,
                        const uint32_t *tau, const uint32_t *nwalks, const Sampler &smp, uint64_t *moments,
                        const PilotParams *pilot, uint32_t *nwalks_out, uint32_t *status, cudaStream_t s) {
    if (k == 0) return BQ_OK;
    if (!edges_uv) return fail(BQ_EINVAL, "pilot moments need explicit edges");
    if (k >= kMaxBucketEdges) return fail(BQ_EINVAL, "k = %llu edges in one pilot", (unsigned long long)k);
    const uint32_t bouquet = 32u * (uint32_t)kMomentW;
    // scratch: info[k] | begin[k + 1] bucket[k + 1] | tasks[k] | next_task
    const size_t info_bytes = sizeof(QueryInfo) * k;
    const size_t begin_bytes = sizeof(uint64_t) * (k + 1) + ((sizeof(uint32_t) * bucket_count(k) + 7) & ~(size_t)7);
    const size_t task_bytes = sizeof(uint32_t) * ((k + 1) & ~1ull);
    char *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, info_bytes + begin_bytes + task_bytes + 16, s);
    if (rc) return rc;
    QueryInfo *info = (QueryInfo *)buf;
    uint64_t *begin = (uint64_t *)(buf + info_bytes);
    uint32_t *tasks = (uint32_t *)(buf + info_bytes + begin_bytes);
    unsigned long long *next_task = (unsigned long long *)(buf + info_bytes + begin_bytes + task_bytes);
    unsigned long long *mo = reinterpret_cast<unsigned long long *>(moments);
    cudaError_t e = cudaMemsetAsync(moments, 0, sizeof(uint64_t) * 10 * k, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next_task, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        scratch_free(buf, s);
        return cuda_fail(e, "pilot setup");
    }
    {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        prepare_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(g, edges_uv, k, tau, nwalks, bouquet, 0u, info,
                                                                    tasks, nullptr, nullptr, status);
        rc = scan_u32_to_u64(tasks, begin, k, s);
        if (rc == BQ_OK) {
            count_launches(1);
            build_bucket_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(
                begin, k, reinterpret_cast<uint32_t *>(begin + k + 1));
        }
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        rc = with_edges(g, [&](auto el) {
            using EL = decltype(el);
            return smp.kind == 1 ? launch_moments<EL, true>(el, g, info, begin, k, seed, smp, next_task, mo, s)
                                 : launch_moments<EL, false>(el, g, info, begin, k, seed, smp, next_task, mo, s);
        });
    }
    if (rc == BQ_OK && pilot) {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        pilot_nwalks_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(info, k, mo, pilot->n0, pilot->eps, pilot->z,
                                                                         pilot->n_min, nwalks_out, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "pilot_nwalks_kernel");
    }
    scratch_free(buf, s);
    return rc;
}

}  // namespace bq
