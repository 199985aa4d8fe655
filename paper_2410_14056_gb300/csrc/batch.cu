// AESC batches: many queries (graphs of uneven sizes, edge subsets or all
// edges) estimated with one persistent counting launch.
//
// The walks, counters and finalize are those of aesc.cu (the walk loop and
// final sum of Alg. 1 at zero push depth): a task is one bouquet of 32*W
// walks of one side of one queried edge.  Here the task space spans all
// queries: a global edge index e runs over the concatenated query edge lists,
// a scan of per-edge task counts maps a task to its edge, and each edge knows
// its query, whose descriptor gives the graph layout and the output buffers.
// bq_batch_run launches kernels only, so it can be captured in a CUDA graph.
#include <math.h>

#include <new>
#include <vector>

#include "edges.cuh"
#include "hash.cuh"
#include "internal.h"

namespace bq {
namespace {

constexpr int kThreads = 256;

// Resident blocks a counting kernel is compiled for: the gathers are latency
// bound, so the common shapes keep 40 warps per SM (<= 48 registers).
template <int W, bool COUPLED>
constexpr int count_min_blocks() {
    return (!COUPLED && W <= 2) ? 6 : ((!COUPLED && W <= 4) ? 5 : 1);
}

__device__ __forceinline__ int64_t lower_bound_row(const uint32_t *__restrict__ nbrs, int64_t lo, int64_t hi,
                                                   uint32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (nbrs[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// largest i in [0, count) with a[i] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ uint64_t last_le(const uint64_t *__restrict__ a, uint64_t count, uint64_t x) {
    uint64_t lo = 0, hi = count;
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Prepare edge i of query d (query index q): normalised endpoints, canonical
// id, degrees and plan into *bi, its task count into *tasks; counters zeroed,
// NaN estimate when the edge is not valid (status bits set).
__device__ __forceinline__ void prepare_edge(const QueryDesc &d, uint64_t i, uint32_t q, uint32_t bouquet,
                                             BInfo *bi_out, uint32_t *tasks_out, uint32_t *status) {
    const GraphDesc &g = d.g;
    uint32_t a, b;
    if (d.uv) {
        a = d.uv[2 * i];
        b = d.uv[2 * i + 1];
    } else {  // canonical edge i: u = last vertex with upper_before[u] <= i
        const uint32_t u = (uint32_t)last_le(g.upper_before, g.n, i);
        const int64_t first = lower_bound_row(g.nbrs, g.offsets[u], g.offsets[u + 1], u + 1);
        a = u;
        b = g.nbrs[first + (int64_t)(i - g.upper_before[u])];
    }
    BInfo bi;
    bi.u = a < b ? a : b;
    bi.v = a < b ? b : a;
    bi.tau = d.tau[i];
    bi.nwalks = d.nwalks[i];
    bi.valid = 0;
    bi.edge = 0;
    bi.du = bi.dv = 0;
    bi.query = q;
    uint32_t bits = 0;
    if (a >= g.n || b >= g.n || a == b) {
        bits = kStatusNoEdge;
    } else {
        const int64_t lo = g.offsets[bi.u], hi = g.offsets[bi.u + 1];
        const int64_t pos = lower_bound_row(g.nbrs, lo, hi, bi.v);
        if (pos >= hi || g.nbrs[pos] != bi.v) {
            bits = kStatusNoEdge;
        } else {
            const int64_t first = lower_bound_row(g.nbrs, lo, hi, bi.u + 1);
            bi.edge = g.upper_before[bi.u] + (uint64_t)(pos - first);
            bi.du = (uint32_t)(hi - lo);
            bi.dv = (uint32_t)(g.offsets[bi.v + 1] - g.offsets[bi.v]);
            if (bi.tau == 0 || bi.nwalks == 0) bits = kStatusBadIndex;
            else if (2ull * bi.nwalks * bi.tau >= (1ull << 32)) bits = kStatusOverflow;
            else bi.valid = 1;
        }
    }
    if (bits) atomicOr(status, bits);
    *bi_out = bi;
    *tasks_out = bi.valid ? 2u * ((bi.nwalks + bouquet - 1) / bouquet) : 0u;
    d.counts[4 * i + 0] = 0u;
    d.counts[4 * i + 1] = 0u;
    d.counts[4 * i + 2] = 0u;
    d.counts[4 * i + 3] = 0u;
    if (!bi.valid) d.sc[i] = __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void batch_prepare_kernel(const QueryDesc *__restrict__ qd, const uint64_t *__restrict__ ebase,
                                     uint32_t nq, uint64_t total, uint32_t bouquet, BInfo *__restrict__ info,
                                     uint32_t *__restrict__ tasks, uint32_t *status) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t q = (uint32_t)last_le(ebase, nq, e);
        prepare_edge(qd[q], e - qd[q].ebase, q, bouquet, info + e, tasks + e, status);
    }
}

// One bouquet task: 32*W walks of one side of one queried edge (`local` =
// task index within the edge: side = local & 1, chunk = local >> 1), the walks
// and counters of aesc_count_kernel; adds the warp's weighted hits to
// d.counts[4 i + 2 side + {0, 1}] (i = the edge's index within its query).
template <typename EL, int W, bool COUPLED>
__device__ __forceinline__ void run_bouquet_task_el(const EL &el, const int64_t *__restrict__ offsets,
                                                    const QueryDesc &d, const BInfo &bi, uint64_t i,
                                                    uint64_t local, const Sampler &smp, uint32_t lane) {
    const uint64_t seed = d.seed;
    const uint32_t side = (uint32_t)(local & 1);
    const uint64_t k0 = (local >> 1) * 32ull * W;
    const uint64_t stream = 2 * bi.edge + side;
    const uint32_t start = side ? bi.v : bi.u;

    uint64_t st[W], gs[W], off[W];
    uint32_t cur[W], deg[W];
    bool act[W];
    if (!COUPLED && (W % 2 == 0)) {
#pragma unroll
        for (int j = 0; j < W; j += 2) {
            const uint64_t kk = k0 + (uint64_t)lane * W + j;
            walk_key_pair(seed, stream, kk >> 1, st[j], st[j + 1]);
            act[j] = kk < bi.nwalks;
            act[j + 1] = kk + 1 < bi.nwalks;
        }
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t kk = COUPLED ? k0 + (uint64_t)j * 32 + lane : k0 + (uint64_t)lane * W + j;
            st[j] = walk_key(seed, stream, kk);
            if (COUPLED) gs[j] = walk_key(seed, stream | kGroupBit, kk / smp.width);
            act[j] = kk < bi.nwalks;
        }
    }
    uint64_t off0;
    uint32_t deg0;
    start_record(offsets, start, off0, deg0);
#pragma unroll
    for (int j = 0; j < W; ++j) {
        cur[j] = start;
        off[j] = off0;
        deg[j] = act[j] ? deg0 : 0u;
        if (!COUPLED) gs[j] = 0;
    }
    uint32_t hit_u = 0, hit_v = 0;
    for (uint32_t l = 1; l <= bi.tau; ++l) {
        const uint32_t weight = l < bi.tau ? 2u : 1u;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            st[j] += kGolden;
            if (COUPLED) gs[j] += kGolden;
            if (deg[j]) {
                const uint32_t kk = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), deg[j]);
                el.next(off[j] + kk, cur[j], off[j], deg[j]);
                hit_u += cur[j] == bi.u ? weight : 0u;
                hit_v += cur[j] == bi.v ? weight : 0u;
            }
        }
    }
#pragma unroll
    for (int dd = 16; dd > 0; dd >>= 1) {
        hit_u += __shfl_down_sync(0xffffffffu, hit_u, dd);
        hit_v += __shfl_down_sync(0xffffffffu, hit_v, dd);
    }
    if (lane == 0) {
        uint32_t *c = d.counts + 4 * i + 2 * side;
        if (hit_u) atomicAdd(c + 0, hit_u);
        if (hit_v) atomicAdd(c + 1, hit_v);
    }
}

// The query's layout is chosen once per task, so each step loop is
// specialised for one layout.
template <int W, bool COUPLED>
__device__ __forceinline__ void run_bouquet_task(const QueryDesc &d, const BInfo &bi, uint64_t i, uint64_t local,
                                                 const Sampler &smp, uint32_t lane) {
    const GraphDesc &g = d.g;
    if (g.edge8) {
        const EdgesPacked el{g.edge8, g.sh_off, g.sh_deg, g.mask_id, g.mask_off};
        run_bouquet_task_el<EdgesPacked, W, COUPLED>(el, g.offsets, d, bi, i, local, smp, lane);
    } else if (g.pk) {
        const EdgesPackedIds el{g.pk, g.rec8, g.pk_bits, g.pk_q, g.pk_mask};
        run_bouquet_task_el<EdgesPackedIds, W, COUPLED>(el, g.offsets, d, bi, i, local, smp, lane);
    } else {
        const EdgesCsr8 el{g.nbrs, g.rec8};
        run_bouquet_task_el<EdgesCsr8, W, COUPLED>(el, g.offsets, d, bi, i, local, smp, lane);
    }
}

// Persistent counting kernel over the tasks of all queries of a batch.
template <int W, bool COUPLED>
__global__ void __launch_bounds__(kThreads, count_min_blocks<W, COUPLED>())
batch_count_kernel(const QueryDesc *__restrict__ qd, const BInfo *__restrict__ info,
                   const uint64_t *__restrict__ begin, const uint32_t *__restrict__ bucket, uint64_t total_edges,
                   Sampler smp, unsigned long long *__restrict__ next_task) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t total = begin[total_edges];
    const uint32_t shift = bucket_shift(total, total_edges);
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const uint64_t e = task_edge(begin, bucket, total_edges, total, shift, t);
        const BInfo bi = info[e];
        const QueryDesc &d = qd[bi.query];
        run_bouquet_task<W, COUPLED>(d, bi, e - d.ebase, t - begin[e], smp, lane);
    }
}

// The server's iteration: windows of several requests' tasks.  Item t ->
// request (items[].item_base) -> its task -> its edge.
template <int W, bool COUPLED>
__global__ void __launch_bounds__(kThreads, count_min_blocks<W, COUPLED>())
serve_count_kernel(const ServeItem *__restrict__ items, uint32_t n_items, uint64_t total_items, Sampler smp,
                   unsigned long long *__restrict__ next_item) {
    const uint32_t lane = threadIdx.x & 31;
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_item, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total_items) break;
        uint32_t lo = 0, hi = n_items;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (items[mid].item_base <= t) lo = mid;
            else hi = mid;
        }
        const ServeItem it = items[lo];
        const uint64_t task = it.task_lo + (t - it.item_base);
        const uint64_t e = last_le_u64(it.begin, 0, it.k, task);
        const BInfo bi = it.info[e];
        run_bouquet_task<W, COUPLED>(*it.qd, bi, e, task - it.begin[e], smp, lane);
    }
}

// Estimate of edge i of query d from its counters (every operation rounded
// to nearest on its own, as the single-query finalize).
__device__ __forceinline__ void finalize_edge(const QueryDesc &d, const BInfo &bi, uint64_t i) {
    const double du = (double)bi.du, dv = (double)bi.dv;
    const double s = __dadd_rn(__ddiv_rn(1.0, du), __ddiv_rn(1.0, dv));
    const uint32_t *c = d.counts + 4 * i;
    const double x = (double)((int64_t)c[0] - (int64_t)c[2]);
    const double y = (double)((int64_t)c[3] - (int64_t)c[1]);
    const double mean = __ddiv_rn(__dadd_rn(__ddiv_rn(x, du), __ddiv_rn(y, dv)), __dmul_rn(2.0, (double)bi.nwalks));
    d.sc[i] = __dadd_rn(s, mean);
}

__global__ void batch_finalize_kernel(const QueryDesc *__restrict__ qd, const BInfo *__restrict__ info,
                                      uint64_t total) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < total;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const BInfo bi = info[e];
        if (!bi.valid) continue;
        const QueryDesc &d = qd[bi.query];
        finalize_edge(d, bi, e - d.ebase);
    }
}

// ------------------------------------------------- server: per-pass launches

// Several requests' prepare, task scan or finalize in one launch; the list
// travels as a kernel parameter.  Request r owns edges [edge_base[r],
// edge_base[r + 1]) of the launch.
__global__ void serve_prepare_many_kernel(ServeMany L, uint32_t bouquet) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < L.edge_base[L.m];
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = 0;
        while (L.edge_base[r + 1] <= e) ++r;
        const uint64_t i = e - L.edge_base[r];
        prepare_edge(*L.qd[r], i, 0, bouquet, L.info[r] + i, L.tasks[r] + i, L.status[r]);
    }
}

// Exclusive scan of request blockIdx.x's task counts into begin[0..k]: one
// block per request, a running carry over tiles of the block's width.
__global__ void __launch_bounds__(1024) serve_scan_many_kernel(ServeMany L) {
    __shared__ uint64_t s_warp[32];
    __shared__ uint64_t s_carry;
    const uint32_t r = blockIdx.x;
    const uint64_t k = L.edge_base[r + 1] - L.edge_base[r];
    const uint32_t *tasks = L.tasks[r];
    uint64_t *begin = L.begin[r];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < k; base += blockDim.x) {
        const uint64_t idx = base + threadIdx.x;
        const uint64_t x = idx < k ? tasks[idx] : 0ull;
        uint64_t incl = x;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t nw = blockDim.x >> 5;
            uint64_t w = lane < nw ? s_warp[lane] : 0ull;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) s_warp[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const uint64_t warp_before = warp ? s_warp[warp - 1] : 0ull;
        const uint64_t carry = s_carry;
        if (idx < k) begin[idx] = carry + warp_before + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + s_warp[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) begin[k] = s_carry;
}

__global__ void serve_finalize_many_kernel(ServeMany L) {
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < L.edge_base[L.m];
         e += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = 0;
        while (L.edge_base[r + 1] <= e) ++r;
        const uint64_t i = e - L.edge_base[r];
        const BInfo bi = L.info[r][i];
        if (bi.valid) finalize_edge(*L.qd[r], bi, i);
    }
}

unsigned blocks_for(uint64_t items, uint64_t per_block) {
    uint64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 0x7fffffffull) b = 0x7fffffffull;
    return (unsigned)b;
}

}  // namespace
}  // namespace bq

struct bq_batch {
    int device = 0;
    uint32_t nq = 0;
    uint64_t edges = 0;
    bq::Sampler smp{0, 0, 1};
    int lanes = 4;
    int grid = 0;
    bq::QueryDesc *d_qd = nullptr;
    uint64_t *d_ebase = nullptr;
    bq::BInfo *d_info = nullptr;
    uint32_t *d_tasks = nullptr;
    uint64_t *d_begin = nullptr;
    uint32_t *d_bucket = nullptr;
    unsigned long long *d_next = nullptr;
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    uint32_t *status = nullptr;
    bq::SharedBatch *shared = nullptr;  // vertex-centric batch (bq_batch_create_shared)
};

using namespace bq;

namespace {

template <int W, bool C>
int batch_occupancy(int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_count_kernel<W, C>, kThreads, 0));
    *grid = sms * (per_sm < 1 ? 1 : per_sm);
    return BQ_OK;
}

template <int W>
void launch_batch_count(const bq_batch *b, cudaStream_t s) {
    if (b->smp.kind == 1)
        batch_count_kernel<W, true><<<b->grid, kThreads, 0, s>>>(b->d_qd, b->d_info, b->d_begin, b->d_bucket,
                                                                 b->edges, b->smp, b->d_next);
    else
        batch_count_kernel<W, false><<<b->grid, kThreads, 0, s>>>(b->d_qd, b->d_info, b->d_begin, b->d_bucket,
                                                                  b->edges, b->smp, b->d_next);
}

void free_batch(bq_batch *b) {
    if (!b) return;
    if (b->shared) shared_batch_free(b->shared);
    cudaFree(b->d_qd);
    cudaFree(b->d_ebase);
    cudaFree(b->d_info);
    cudaFree(b->d_tasks);
    cudaFree(b->d_begin);
    cudaFree(b->d_bucket);
    cudaFree(b->d_next);
    cudaFree(b->d_ws);
    delete b;
}

}  // namespace

extern "C" {

int bq_batch_create(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler, bq_batch **out) {
    bq::NvtxRange nvtx_range("bq_batch_create");
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_queries == 0 || !queries) return fail(BQ_EINVAL, "a batch needs at least one query");
    Sampler smp;
    int rc = validate_sampler(sampler, smp);
    if (rc) return rc;
    int dev = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    std::vector<QueryDesc> qd(n_queries);
    std::vector<uint64_t> ebase(n_queries + 1, 0);
    uint64_t total = 0;
    for (uint32_t q = 0; q < n_queries; ++q) {
        const bq_aesc_query &in = queries[q];
        const bq_graph *g = in.graph;
        if (!g) return fail(BQ_EINVAL, "query %u: graph is NULL", q);
        if (g->device != dev) return fail(BQ_EINVAL, "query %u: graph lives on device %d, not %d", q, g->device, dev);
        if (!g->d_rec8) return fail(BQ_EINVAL, "query %u: batches need graphs with nnz < 2^32", q);
        if (in.k && (!in.tau_dev || !in.nwalks_dev || !in.counts_dev || !in.sc_dev))
            return fail(BQ_EINVAL, "query %u: tau, nwalks, counts or sc is NULL", q);
        if (!in.edges_uv_dev && (in.k != g->nnz / 2 || in.k != g->m_upper))
            return fail(BQ_EINVAL, "query %u: all-edges query needs k = m = %llu", q,
                        (unsigned long long)(g->nnz / 2));
        QueryDesc &d = qd[q];
        const DeviceGraph v = g->view();
        d.g.offsets = v.offsets;
        d.g.nbrs = v.nbrs;
        d.g.rec8 = v.rec8;
        d.g.upper_before = v.upper_before;
        d.g.pk = v.pk;
        d.g.edge8 = v.edge8;
        d.g.mask_off = v.mask_off;
        d.g.n = v.n;
        d.g.pk_bits = v.pk_bits;
        d.g.pk_q = v.pk_q;
        d.g.pk_mask = v.pk_mask;
        d.g.sh_off = v.sh_off;
        d.g.sh_deg = v.sh_deg;
        d.g.mask_id = v.mask_id;
        d.g.pad = 0;
        d.seed = in.seed;
        d.uv = in.edges_uv_dev;
        d.tau = in.tau_dev;
        d.nwalks = in.nwalks_dev;
        d.counts = in.counts_dev;
        d.sc = in.sc_dev;
        d.k = in.k;
        d.ebase = total;
        ebase[q] = total;
        total += in.k;
    }
    ebase[n_queries] = total;
    uint32_t *status = nullptr;
    rc = status_word(dev, &status);
    if (rc) return rc;
    bq_batch *b = new (std::nothrow) bq_batch();
    if (!b) return fail(BQ_ENOMEM, "host allocation failed");
    b->device = dev;
    b->nq = n_queries;
    b->edges = total;
    b->smp = smp;
    b->status = status;
    if (total >= kMaxBucketEdges) {
        delete b;
        return fail(BQ_EINVAL, "a batch of %llu edges (at most 2^32 - 2)", (unsigned long long)total);
    }
    b->lanes = tuning_aesc_walks_per_lane();
    if (b->lanes != 2 && b->lanes != 8) b->lanes = 4;
    b->ws_bytes = scan_u32_to_u64_ws_bytes(total);
    cudaError_t e = cudaMalloc(&b->d_qd, sizeof(QueryDesc) * n_queries);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_ebase, sizeof(uint64_t) * (n_queries + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_info, sizeof(BInfo) * (total ? total : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_tasks, sizeof(uint32_t) * (total ? total : 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_begin, sizeof(uint64_t) * (total + 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bucket, sizeof(uint32_t) * bucket_count(total));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned long long));
    if (e == cudaSuccess && b->ws_bytes) e = cudaMalloc(&b->d_ws, b->ws_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_qd, qd.data(), sizeof(QueryDesc) * n_queries, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_ebase, ebase.data(), sizeof(uint64_t) * (n_queries + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(b);
        return e == cudaErrorMemoryAllocation ? fail(BQ_ENOMEM, "cannot allocate the batch buffers")
                                              : cuda_fail(e, "bq_batch_create");
    }
    const bool c = smp.kind == 1;
    rc = b->lanes == 2 ? (c ? batch_occupancy<2, true>(&b->grid) : batch_occupancy<2, false>(&b->grid))
       : b->lanes == 8 ? (c ? batch_occupancy<8, true>(&b->grid) : batch_occupancy<8, false>(&b->grid))
                       : (c ? batch_occupancy<4, true>(&b->grid) : batch_occupancy<4, false>(&b->grid));
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return BQ_OK;
}

int bq_batch_create_shared(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler,
                           bq_batch **out) {
    bq::NvtxRange nvtx_range("bq_batch_create_shared");
    clear_error();
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_queries == 0 || !queries) return fail(BQ_EINVAL, "a batch needs at least one query");
    Sampler smp;
    int rc = validate_sampler(sampler, smp);
    if (rc) return rc;
    bq_batch *b = new (std::nothrow) bq_batch();
    if (!b) return fail(BQ_ENOMEM, "host allocation failed");
    BQ_CUDA(cudaGetDevice(&b->device));
    b->nq = n_queries;
    b->smp = smp;
    rc = shared_batch_create(queries, n_queries, smp, &b->shared, &b->edges);
    if (rc) {
        delete b;
        return rc;
    }
    *out = b;
    return BQ_OK;
}

int bq_batch_run(bq_batch *b, void *stream) {
    bq::NvtxRange nvtx_range("bq_batch_run");
    if (!b) return fail(BQ_EINVAL, "batch is NULL");
    if (b->edges == 0) return BQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != b->device) cudaSetDevice(b->device);
    if (b->shared) {
        const int rc = shared_batch_run(b->shared, s);
        if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
        return rc;
    }
    const uint32_t bouquet = 32u * (uint32_t)b->lanes;
    int rc = BQ_OK;
    cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) rc = cuda_fail(e, "bq_batch_run");
    if (rc == BQ_OK) {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        batch_prepare_kernel<<<blocks_for(b->edges, kThreads), kThreads, 0, s>>>(
            b->d_qd, b->d_ebase, b->nq, b->edges, bouquet, b->d_info, b->d_tasks, b->status);
        rc = scan_u32_to_u64_ws(b->d_tasks, b->d_begin, b->edges, b->d_ws, b->ws_bytes, s);
        if (rc == BQ_OK) {
            count_launches(1);
            build_bucket_kernel<<<blocks_for(b->edges, kThreads), kThreads, 0, s>>>(b->d_begin, b->edges,
                                                                                   b->d_bucket);
        }
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        if (b->lanes == 2) launch_batch_count<2>(b, s);
        else if (b->lanes == 8) launch_batch_count<8>(b, s);
        else launch_batch_count<4>(b, s);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "batch_count_kernel");
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        batch_finalize_kernel<<<blocks_for(b->edges, kThreads), kThreads, 0, s>>>(b->d_qd, b->d_info, b->edges);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "batch_finalize_kernel");
    }
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
}

int bq_batch_size(const bq_batch *b, uint64_t *edges) {
    if (!b || !edges) return fail(BQ_EINVAL, "NULL argument");
    *edges = b->edges;
    return BQ_OK;
}

int bq_batch_destroy(bq_batch *b) {
    if (!b) return BQ_OK;
    const int device = b->device;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != device) cudaSetDevice(device);
    free_batch(b);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return BQ_OK;
}

}  // extern "C"

// ------------------------------------------------------------ server hooks

namespace bq {

GraphDesc graph_desc(const bq_graph *g) {
    const DeviceGraph v = g->view();
    GraphDesc d;
    d.offsets = v.offsets;
    d.nbrs = v.nbrs;
    d.rec8 = v.rec8;
    d.upper_before = v.upper_before;
    d.pk = v.pk;
    d.edge8 = v.edge8;
    d.mask_off = v.mask_off;
    d.n = v.n;
    d.pk_bits = v.pk_bits;
    d.pk_q = v.pk_q;
    d.pk_mask = v.pk_mask;
    d.sh_off = v.sh_off;
    d.sh_deg = v.sh_deg;
    d.mask_id = v.mask_id;
    d.pad = 0;
    return d;
}


// Persistent grid of a serve_count_kernel shape (SMs x resident blocks),
// taken once per process: every iteration of a server launches it.
template <int W, bool COUPLED>
int serve_grid() {
    static const int grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_count_kernel<W, COUPLED>, kThreads, 0) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return sms * (per_sm < 1 ? 1 : per_sm);
    }();
    return grid;
}

template <int W, bool COUPLED>
int launch_serve(const ServeItem *d_items, uint32_t n_items, uint64_t total_items, const Sampler &smp,
                 unsigned long long *counter, cudaStream_t s) {
    const int grid = serve_grid<W, COUPLED>();
    if (grid <= 0) return fail(BQ_ECUDA, "serve_count_kernel: no launch configuration");
    serve_count_kernel<W, COUPLED><<<grid, kThreads, 0, s>>>(d_items, n_items, total_items, smp, counter);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

int serve_iterate(const ServeItem *d_items, uint32_t n_items, uint64_t total_items, int lanes, const Sampler &smp,
                  unsigned long long *counter, cudaStream_t s) {
    if (total_items == 0) return BQ_OK;
    BQ_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    const bool c = smp.kind == 1;
    ProfScope prof(kProfAesc, s);
    count_launches(1);
    if (lanes == 2) return c ? launch_serve<2, true>(d_items, n_items, total_items, smp, counter, s)
                             : launch_serve<2, false>(d_items, n_items, total_items, smp, counter, s);
    if (lanes == 8) return c ? launch_serve<8, true>(d_items, n_items, total_items, smp, counter, s)
                             : launch_serve<8, false>(d_items, n_items, total_items, smp, counter, s);
    return c ? launch_serve<4, true>(d_items, n_items, total_items, smp, counter, s)
             : launch_serve<4, false>(d_items, n_items, total_items, smp, counter, s);
}

int serve_prepare_many(const ServeMany &L, uint32_t bouquet, cudaStream_t s) {
    if (L.m == 0) return BQ_OK;
    const uint64_t edges = L.edge_base[L.m];
    if (edges) {
        count_launches(1);
        serve_prepare_many_kernel<<<blocks_for(edges, kThreads), kThreads, 0, s>>>(L, bouquet);
        BQ_CUDA(cudaGetLastError());
    }
    count_launches(1);
    serve_scan_many_kernel<<<L.m, 1024, 0, s>>>(L);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

int serve_finalize_many(const ServeMany &L, cudaStream_t s) {
    const uint64_t edges = L.m ? L.edge_base[L.m] : 0;
    if (edges == 0) return BQ_OK;
    count_launches(1);
    serve_finalize_many_kernel<<<blocks_for(edges, kThreads), kThreads, 0, s>>>(L);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}


}  // namespace bq
