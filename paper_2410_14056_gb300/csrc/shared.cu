// Vertex-centric AESC: the walk loop of TGT+ (Alg. 1) with the walks of a
// vertex shared by every query edge at that vertex.
//
// Every endpoint x of a query edge runs N_x = max nwalks and tau_x = max tau
// over the query edges at x (walk w < N_x keyed on stream kVertexStream | x).
// A walk from x standing on x at step l counts a return, kept per (x, l) in a
// histogram so that each edge weighs the returns by its own tau; a walk from x
// standing on a query neighbour y of x at step l <= tau of {x, y} adds that
// step's weight (2 before tau, 1 at tau) to the edge's cross counter.  The
// neighbour test is one binary search of y in x's row, which every walk of a
// task shares (L1-resident), and a per-CSR-position query index maps the hit
// to its edge, so no query list is sorted.
//
// Work decomposition (GB300): a task is a bouquet of 32*W walks of one vertex
// (Alg. 3 with B = 32*W); a persistent grid of warps pulls tasks through the
// bucket index of the vertices' task prefix.  Returns are counted with a
// ballot per step and lane; cross hits are combined across the warp with
// match.any on the edge before one atomic per distinct edge.
#include <math.h>

#include <new>
#include <vector>

#include "edges.cuh"
#include "hash.cuh"
#include "internal.h"

namespace bq {
namespace {

constexpr int kThreads = 256;
constexpr int kSharedW = 2;                                 // walks per lane (coupled sampler)
constexpr uint64_t kVertexStream = 0x2000000000000000ull;  // edge streams stay below
constexpr uint32_t kNoQuery = 0xffffffffu;

struct SharedQuery {
    uint32_t u, v;  // normalised endpoints, u < v
    uint32_t tau, nwalks;
    uint32_t valid;
    uint32_t pad;
};

unsigned blocks_for(uint64_t items, uint64_t per_block) {
    uint64_t b = (items + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 0x7fffffffull) b = 0x7fffffffull;
    return (unsigned)b;
}

// first index in [lo, hi) whose entry is >= key
__device__ __forceinline__ int64_t lower_bound_ids(const uint32_t *__restrict__ nbrs, int64_t lo, int64_t hi,
                                                   uint32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(nbrs + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Validate the queries, take the per-vertex maxima of N and tau, and claim
// the two CSR positions of each edge in the query index (a second claim of
// the same position is a repeated edge).
__global__ void shared_prepare_kernel(DeviceGraph g, const uint32_t *__restrict__ uv, uint64_t k,
                                      const uint32_t *__restrict__ tau, const uint32_t *__restrict__ nwalks,
                                      SharedQuery *__restrict__ qinfo, uint32_t *__restrict__ vn,
                                      uint32_t *__restrict__ vt, uint32_t *__restrict__ qidx, uint32_t *status) {
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        SharedQuery qi;
        const uint32_t a = uv[2 * q], b = uv[2 * q + 1];
        qi.u = a < b ? a : b;
        qi.v = a < b ? b : a;
        qi.tau = tau[q];
        qi.nwalks = nwalks[q];
        qi.valid = 0;
        qi.pad = 0;
        uint32_t bits = 0;
        if (a >= g.n || b >= g.n || a == b) {
            bits = kStatusNoEdge;
        } else {
            const int64_t lu = g.offsets[qi.u], hu = g.offsets[qi.u + 1];
            const int64_t lv = g.offsets[qi.v], hv = g.offsets[qi.v + 1];
            const int64_t puv = lower_bound_ids(g.nbrs, lu, hu, qi.v);
            const int64_t pvu = lower_bound_ids(g.nbrs, lv, hv, qi.u);
            if (puv >= hu || g.nbrs[puv] != qi.v || pvu >= hv || g.nbrs[pvu] != qi.u) {
                bits = kStatusNoEdge;
            } else if (qi.tau == 0 || qi.nwalks == 0) {
                bits = kStatusBadIndex;
            } else if (atomicCAS(qidx + puv, kNoQuery, (uint32_t)q) != kNoQuery) {
                bits = kStatusRepeated;
            } else {
                qidx[pvu] = (uint32_t)q;
                qi.valid = 1;
                atomicMax(vn + qi.u, qi.nwalks);
                atomicMax(vn + qi.v, qi.nwalks);
                atomicMax(vt + qi.u, qi.tau);
                atomicMax(vt + qi.v, qi.tau);
            }
        }
        if (bits) atomicOr(status, bits);
        qinfo[q] = qi;
    }
}

__global__ void vertex_tasks_kernel(uint64_t n, const uint32_t *__restrict__ vn, uint32_t bouquet,
                                    uint32_t *__restrict__ tasks) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        tasks[x] = (vn[x] + bouquet - 1) / bouquet;
}

// One vertex task: walks [k0, k0 + 32 W) of vertex x (of its nx walks, tx
// steps each, keyed on stream kVertexStream | x), run by a whole warp.
// Returns at step l go to ret[rb + l - 1] (one atomic per step for the
// warp; entries at or past ret_cap are never written), cross hits to
// cross[2 q + side] (one atomic per distinct edge side and step).
template <typename EL, int W, bool COUPLED>
__device__ __forceinline__ void run_vertex_task(const EL &el, const int64_t *__restrict__ offsets,
                                                const uint32_t *__restrict__ nbrs, uint32_t x, uint64_t k0,
                                                uint32_t nx, uint32_t tx, uint64_t rb, uint64_t ret_cap,
                                                const uint32_t *__restrict__ qidx,
                                                const SharedQuery *__restrict__ qinfo, uint64_t seed,
                                                const Sampler &smp, uint32_t *__restrict__ ret,
                                                uint32_t *__restrict__ cross, uint32_t lane) {
    const uint64_t stream = kVertexStream | x;
    uint64_t st[W], gs[W];
    bool act[W];
    if (!COUPLED && (W % 2 == 0)) {
#pragma unroll
        for (int j = 0; j < W; j += 2) {
            const uint64_t kk = k0 + (uint64_t)lane * W + j;
            walk_key_pair(seed, stream, kk >> 1, st[j], st[j + 1]);
            act[j] = kk < nx;
            act[j + 1] = kk + 1 < nx;
            gs[j] = gs[j + 1] = 0;
        }
    } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const uint64_t kk = COUPLED ? k0 + (uint64_t)j * 32 + lane : k0 + (uint64_t)lane * W + j;
            st[j] = walk_key(seed, stream, kk);
            gs[j] = COUPLED ? walk_key(seed, stream | kGroupBit, kk / smp.width) : 0;
            act[j] = kk < nx;
        }
    }
    uint64_t off0;
    uint32_t deg0;
    start_record(offsets, x, off0, deg0);
    const uint32_t *__restrict__ row = nbrs + off0;  // the start's row and its query index
    const uint32_t *__restrict__ qrow = qidx + off0;
    uint64_t off[W];
    uint32_t cur[W], deg[W];
#pragma unroll
    for (int j = 0; j < W; ++j) {
        cur[j] = x;
        off[j] = off0;
        deg[j] = act[j] ? deg0 : 0u;  // inactive walks never move or hit
    }
    for (uint32_t l = 1; l <= tx; ++l) {
        uint32_t returns = 0;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            st[j] += kGolden;
            if (COUPLED) gs[j] += kGolden;
            uint32_t key = kNoQuery, w = 0;
            if (deg[j]) {
                const bool from_x = cur[j] == x;
                const uint32_t kk = choose(sample_word<COUPLED>(st[j], gs[j], cur[j], smp.t), deg[j]);
                el.next(off[j] + kk, cur[j], off[j], deg[j]);
                if (cur[j] != x) {
                    // a step taken from x lands on position kk of x's row;
                    // any other step searches the row for the new vertex
                    uint32_t p = kk;
                    bool in_row = from_x;
                    if (!from_x) {
                        p = last_le_row(row, deg0, cur[j]);
                        in_row = __ldg(row + p) == cur[j];
                    }
                    if (in_row) {
                        const uint32_t q = __ldg(qrow + p);
                        if (q != kNoQuery) {
                            const uint32_t tq = qinfo[q].tau;
                            if (l <= tq) {
                                key = 2 * q + (x < cur[j] ? 0u : 1u);
                                w = l < tq ? 2u : 1u;
                            }
                        }
                    }
                }
            }
            returns += __popc(__ballot_sync(0xffffffffu, deg[j] != 0 && cur[j] == x));
            // lanes hitting the same edge side at this step share one atomic
            // (the match is skipped when no lane hit a query neighbour)
            if (__any_sync(0xffffffffu, key != kNoQuery)) {
                const uint32_t peers = __match_any_sync(0xffffffffu, key);
                if (key != kNoQuery && lane == (uint32_t)(__ffs(peers) - 1))
                    atomicAdd(cross + key, w * (uint32_t)__popc(peers));
            }
        }
        if (lane == 0 && returns && rb + (l - 1) < ret_cap) atomicAdd(ret + rb + (l - 1), returns);
    }
}

template <typename EL, int W, bool COUPLED>
__global__ void __launch_bounds__(kThreads)
shared_count_kernel(EL el, const int64_t *__restrict__ offsets, const uint32_t *__restrict__ nbrs,
                    const uint32_t *__restrict__ vn, const uint32_t *__restrict__ vt,
                    const uint64_t *__restrict__ vbegin, const uint32_t *__restrict__ bucket, uint64_t n,
                    const uint64_t *__restrict__ rbegin, uint64_t ret_cap, const uint32_t *__restrict__ qidx,
                    const SharedQuery *__restrict__ qinfo, uint64_t seed, Sampler smp,
                    unsigned long long *__restrict__ next_task, uint32_t *__restrict__ ret,
                    uint32_t *__restrict__ cross) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t total = vbegin[n];
    const uint32_t shift = bucket_shift(total, n);
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        const uint32_t x = (uint32_t)task_edge(vbegin, bucket, n, total, shift, t);
        const uint64_t k0 = (t - vbegin[x]) * 32ull * W;
        run_vertex_task<EL, W, COUPLED>(el, offsets, nbrs, x, k0, vn[x], vt[x], rbegin[x], ret_cap, qidx, qinfo,
                                        seed, smp, ret, cross, lane);
    }
}

// Counters and estimate per query: C_uu and C_vv from the return histograms
// of u and v weighted by the edge's own tau, C_uv and C_vu from the cross
// counters; est = s_e + ((C_uu/N_u - C_vu/N_v)/d_u + (C_vv/N_v - C_uv/N_u)/d_v)/2,
// every operation rounded on its own (_rn intrinsics).
// A plan whose histograms need more than ret_cap entries (possible only in
// a batch whose plan grew after creation) gives NaN and BQ_EINVAL.
__global__ void shared_finalize_kernel(const SharedQuery *__restrict__ qinfo, uint64_t k,
                                       const int64_t *__restrict__ offsets, const uint32_t *__restrict__ vn,
                                       const uint64_t *__restrict__ rbegin, uint64_t n, uint64_t ret_cap,
                                       const uint32_t *__restrict__ ret, const uint32_t *__restrict__ cross,
                                       uint32_t *__restrict__ counts, uint32_t *__restrict__ nused,
                                       double *__restrict__ sc, uint32_t *status) {
    const bool fits = rbegin[n] <= ret_cap;
    if (!fits && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusPlanGrew);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < k;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const SharedQuery qi = qinfo[q];
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        if (!qi.valid || !fits) {
            sc[q] = nan;
            continue;
        }
        const uint32_t nu = vn[qi.u], nv = vn[qi.v];
        if (2ull * (nu > nv ? nu : nv) * qi.tau >= (1ull << 32)) {
            atomicOr(status, kStatusOverflow);
            sc[q] = nan;
            continue;
        }
        uint64_t cuu = 0, cvv = 0;
        const uint32_t *ru = ret + rbegin[qi.u], *rv = ret + rbegin[qi.v];
        for (uint32_t l = 1; l <= qi.tau; ++l) {
            const uint32_t w = l < qi.tau ? 2u : 1u;
            cuu += (uint64_t)w * ru[l - 1];
            cvv += (uint64_t)w * rv[l - 1];
        }
        const uint32_t cuv = cross[2 * q], cvu = cross[2 * q + 1];
        counts[4 * q + 0] = (uint32_t)cuu;
        counts[4 * q + 1] = cuv;
        counts[4 * q + 2] = cvu;
        counts[4 * q + 3] = (uint32_t)cvv;
        if (nused) {
            nused[2 * q] = nu;
            nused[2 * q + 1] = nv;
        }
        const double du = (double)(offsets[qi.u + 1] - offsets[qi.u]);
        const double dv = (double)(offsets[qi.v + 1] - offsets[qi.v]);
        const double s = __dadd_rn(__ddiv_rn(1.0, du), __ddiv_rn(1.0, dv));
        const double fu = (double)nu, fv = (double)nv;
        const double ruu = __ddiv_rn((double)cuu, fu), ruv = __ddiv_rn((double)cuv, fu);
        const double rvu = __ddiv_rn((double)cvu, fv), rvv = __ddiv_rn((double)cvv, fv);
        const double mean =
            __ddiv_rn(__dadd_rn(__ddiv_rn(__dsub_rn(ruu, rvu), du), __ddiv_rn(__dsub_rn(rvv, ruv), dv)), 2.0);
        sc[q] = __dadd_rn(s, mean);
    }
}

// Walks per lane of the vertex-centric kernels (bq_tuning.shared_lanes; the
// coupled sampler keeps kSharedW): never changes a result, the walks of a
// vertex are the same whatever their grouping.
int shared_walks_per_lane(const Sampler &smp) {
    const int w = tuning_shared_lanes();
    return smp.kind == 1 || (w != 2 && w != 4 && w != 8) ? kSharedW : w;
}

template <typename EL, int W, bool COUPLED>
int launch_shared_count(EL el, const DeviceGraph &g, const uint32_t *vn, const uint32_t *vt, const uint64_t *vbegin,
                        const uint32_t *bucket, const uint64_t *rbegin, uint64_t ret_cap, const uint32_t *qidx,
                        const SharedQuery *qinfo, uint64_t seed, const Sampler &smp,
                        unsigned long long *next_task, uint32_t *ret, uint32_t *cross, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kernel = shared_count_kernel<EL, W, COUPLED>;
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    kernel<<<sms * per_sm, kThreads, 0, s>>>(el, g.offsets, g.nbrs, vn, vt, vbegin, bucket, g.n, rbegin, ret_cap,
                                             qidx, qinfo, seed, smp, next_task, ret, cross);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

}  // namespace

namespace {

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

// Asynchronous on s except for one wait, after the per-vertex plan, that
// reads the length of the return histograms to size them.
int launch_aesc_shared(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k,
                       const uint32_t *tau, const uint32_t *nwalks, const Sampler &smp, uint32_t *counts,
                       uint32_t *nused, double *sc, uint32_t *status, cudaStream_t s) {
    if (k == 0) return BQ_OK;
    const uint64_t n = g.n;
    const int lanes_w = shared_walks_per_lane(smp);
    const uint32_t bouquet = 32u * (uint32_t)lanes_w;
    // scratch: qinfo[k] | vn[n] vt[n] | tasks[n] | vbegin[n + 1] bucket | rbegin[n + 1] |
    // qidx[nnz] | cross[2k] | next_task | (edges[2k] if all-edges)
    const size_t b_qinfo = align16(sizeof(SharedQuery) * k);
    const size_t b_vnt = align16(sizeof(uint32_t) * 2 * n);
    const size_t b_tasks = align16(sizeof(uint32_t) * n);
    const size_t b_vbegin = align16(sizeof(uint64_t) * (n + 1) + sizeof(uint32_t) * bucket_count(n));
    const size_t b_rbegin = align16(sizeof(uint64_t) * (n + 1));
    const size_t b_qidx = align16(sizeof(uint32_t) * g.nnz);
    const size_t b_cross = align16(sizeof(uint32_t) * 2 * k);
    const size_t b_edges = edges_uv ? 0 : align16(sizeof(uint32_t) * 2 * k);
    const size_t bytes = b_qinfo + b_vnt + b_tasks + b_vbegin + b_rbegin + b_qidx + b_cross + 16 + b_edges;
    char *buf = nullptr;
    int rc = scratch_alloc((void **)&buf, bytes, s);
    if (rc) return rc;
    char *p = buf;
    SharedQuery *qinfo = (SharedQuery *)p;
    p += b_qinfo;
    uint32_t *vn = (uint32_t *)p;
    uint32_t *vt = vn + n;
    p += b_vnt;
    uint32_t *tasks = (uint32_t *)p;
    p += b_tasks;
    uint64_t *vbegin = (uint64_t *)p;
    uint32_t *bucket = (uint32_t *)(vbegin + n + 1);
    p += b_vbegin;
    uint64_t *rbegin = (uint64_t *)p;
    p += b_rbegin;
    uint32_t *qidx = (uint32_t *)p;
    p += b_qidx;
    uint32_t *cross = (uint32_t *)p;
    p += b_cross;
    unsigned long long *next_task = (unsigned long long *)p;
    p += 16;
    uint32_t *all_uv = edges_uv ? nullptr : (uint32_t *)p;

    cudaError_t e = cudaMemsetAsync(vn, 0, sizeof(uint32_t) * 2 * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(qidx, 0xff, sizeof(uint32_t) * g.nnz, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cross, 0, sizeof(uint32_t) * 2 * k, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(next_task, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        scratch_free(buf, s);
        return cuda_fail(e, "shared setup");
    }
    const uint32_t *uv = edges_uv;
    uint64_t ret_len = 0;
    {
        ProfScope prof(kProfAescAux, s);
        if (!uv) {
            rc = launch_canonical_edges(g, all_uv, s);
            uv = all_uv;
        }
        if (rc == BQ_OK) {
            count_launches(2);
            shared_prepare_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(g, uv, k, tau, nwalks, qinfo, vn, vt,
                                                                               qidx, status);
            vertex_tasks_kernel<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, vn, bouquet, tasks);
            rc = scan_u32_to_u64(tasks, vbegin, n, s);
        }
        if (rc == BQ_OK) {
            count_launches(1);
            build_bucket_kernel<<<blocks_for(n, kThreads), kThreads, 0, s>>>(vbegin, n, bucket);
            rc = scan_u32_to_u64(vt, rbegin, n, s);
        }
        if (rc == BQ_OK) {
            e = cudaMemcpyAsync(&ret_len, rbegin + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = cuda_fail(e, "shared plan");
        }
    }
    uint32_t *ret = nullptr;
    if (rc == BQ_OK) rc = scratch_alloc((void **)&ret, sizeof(uint32_t) * (ret_len + 1), s);
    if (rc == BQ_OK) {
        e = cudaMemsetAsync(ret, 0, sizeof(uint32_t) * (ret_len + 1), s);
        if (e != cudaSuccess) rc = cuda_fail(e, "shared histogram");
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        rc = with_edges(g, [&](auto el) {
            using EL = decltype(el);
            if (smp.kind == 1)
                return launch_shared_count<EL, kSharedW, true>(el, g, vn, vt, vbegin, bucket, rbegin, ret_len + 1,
                                                               qidx, qinfo, seed, smp, next_task, ret, cross, s);
            if (lanes_w == 4)
                return launch_shared_count<EL, 4, false>(el, g, vn, vt, vbegin, bucket, rbegin, ret_len + 1, qidx,
                                                         qinfo, seed, smp, next_task, ret, cross, s);
            if (lanes_w == 8)
                return launch_shared_count<EL, 8, false>(el, g, vn, vt, vbegin, bucket, rbegin, ret_len + 1, qidx,
                                                         qinfo, seed, smp, next_task, ret, cross, s);
            return launch_shared_count<EL, 2, false>(el, g, vn, vt, vbegin, bucket, rbegin, ret_len + 1, qidx,
                                                     qinfo, seed, smp, next_task, ret, cross, s);
        });
    }
    if (rc == BQ_OK) {
        ProfScope prof(kProfAescAux, s);
        count_launches(1);
        shared_finalize_kernel<<<blocks_for(k, kThreads), kThreads, 0, s>>>(qinfo, k, g.offsets, vn, rbegin, n,
                                                                            ret_len + 1, ret, cross, counts, nused,
                                                                            sc, status);
        e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "shared_finalize_kernel");
    }
    if (ret) scratch_free(ret, s);
    scratch_free(buf, s);
    return rc;
}

// ------------------------------------------------------------ batches
//
// Many vertex-centric estimates (graphs of uneven sizes, subsets or all
// edges) in one batch: each query keeps its own per-vertex plan (walk counts,
// lengths, task prefix, return histograms, query index), built by the same
// kernels as a single call, and one persistent launch runs the vertex tasks
// of every query.  A global task t belongs to the last query q with
// qbase[q] <= t; within q it is found through q's bucket index.  Each query's
// counters and estimates are those of bq_aesc_estimate_shared on it alone.

namespace {

struct SharedQueryDesc {
    GraphDesc g;
    uint64_t seed;
    uint64_t n;
    const uint32_t *vn, *vt;
    const uint64_t *vbegin;
    const uint32_t *bucket;
    const uint64_t *rbegin;
    const uint32_t *qidx;
    const SharedQuery *qinfo;
    uint32_t *ret;
    uint32_t *cross;
    uint64_t ret_cap;
};

// qbase[q] = tasks of the queries before q (one thread: a few hundred queries)
__global__ void shared_qbase_kernel(const SharedQueryDesc *__restrict__ qd, uint32_t nq, uint64_t *__restrict__ qbase) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    uint64_t acc = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        qbase[q] = acc;
        acc += qd[q].vbegin[qd[q].n];
    }
    qbase[nq] = acc;
}

// 6 resident blocks at 2 walks per lane (40 registers instead of 46, 48 warps
// instead of 40): measured 2.4 % faster on a 48-graph batch.
template <int W, bool COUPLED>
__global__ void __launch_bounds__(kThreads, (!COUPLED && W <= 2) ? 6 : 1)
shared_batch_count_kernel(const SharedQueryDesc *__restrict__ qd, const uint64_t *__restrict__ qbase, uint32_t nq,
                          Sampler smp, unsigned long long *__restrict__ next_task) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t total = qbase[nq];
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(next_task, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        uint32_t lo = 0, hi = nq;  // the last q with qbase[q] <= t (it has tasks)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (qbase[mid] <= t) lo = mid;
            else hi = mid;
        }
        const SharedQueryDesc &d = qd[lo];
        const uint64_t tl = t - qbase[lo];
        const uint64_t qtotal = d.vbegin[d.n];
        const uint32_t x = (uint32_t)task_edge(d.vbegin, d.bucket, d.n, qtotal, bucket_shift(qtotal, d.n), tl);
        const uint64_t k0 = (tl - d.vbegin[x]) * 32ull * W;
        const GraphDesc &g = d.g;
        if (g.edge8) {
            const EdgesPacked el{g.edge8, g.sh_off, g.sh_deg, g.mask_id, g.mask_off};
            run_vertex_task<EdgesPacked, W, COUPLED>(el, g.offsets, g.nbrs, x, k0, d.vn[x], d.vt[x], d.rbegin[x],
                                                     d.ret_cap, d.qidx, d.qinfo, d.seed, smp, d.ret, d.cross, lane);
        } else if (g.pk) {
            const EdgesPackedIds el{g.pk, g.rec8, g.pk_bits, g.pk_q, g.pk_mask};
            run_vertex_task<EdgesPackedIds, W, COUPLED>(el, g.offsets, g.nbrs, x, k0, d.vn[x], d.vt[x], d.rbegin[x],
                                                        d.ret_cap, d.qidx, d.qinfo, d.seed, smp, d.ret, d.cross,
                                                        lane);
        } else {
            const EdgesCsr8 el{g.nbrs, g.rec8};
            run_vertex_task<EdgesCsr8, W, COUPLED>(el, g.offsets, g.nbrs, x, k0, d.vn[x], d.vt[x], d.rbegin[x],
                                                   d.ret_cap, d.qidx, d.qinfo, d.seed, smp, d.ret, d.cross, lane);
        }
    }
}

}  // namespace

struct SharedBatchQuery {
    DeviceGraph g;
    uint64_t seed = 0, k = 0;
    const uint32_t *uv = nullptr;  // the caller's pairs, or own_uv (all edges)
    const uint32_t *tau = nullptr, *nwalks = nullptr;
    uint32_t *counts = nullptr;
    double *sc = nullptr;
    uint32_t *own_uv = nullptr;
    char *buf = nullptr;  // qinfo | vn vt | tasks | vbegin bucket | rbegin | qidx | cross | scan workspace
    uint32_t *ret = nullptr;
    SharedQuery *qinfo = nullptr;
    uint32_t *vn = nullptr, *vt = nullptr, *tasks = nullptr, *bucket = nullptr, *qidx = nullptr, *cross = nullptr;
    uint64_t *vbegin = nullptr, *rbegin = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    uint64_t ret_cap = 0;
};

struct SharedBatch {
    int device = 0;
    Sampler smp{0, 0, 1};
    int lanes = kSharedW;  // walks per lane, fixed at creation
    uint64_t edges = 0;
    int grid = 0;
    std::vector<SharedBatchQuery> q;
    SharedQueryDesc *d_qd = nullptr;
    uint64_t *d_qbase = nullptr;
    unsigned long long *d_next = nullptr;
    uint32_t *status = nullptr;
};

void shared_batch_free_impl(SharedBatch *b) {
    if (!b) return;
    for (SharedBatchQuery &q : b->q) {
        cudaFree(q.own_uv);
        cudaFree(q.buf);
        cudaFree(q.ret);
    }
    cudaFree(b->d_qd);
    cudaFree(b->d_qbase);
    cudaFree(b->d_next);
    delete b;
}

// The per-vertex plan of one query on s (the first half of a single call):
// validation, walk counts and lengths, vertex task prefix and bucket index,
// histogram offsets; zeroes the return histograms it will fill.
int shared_plan(const SharedBatchQuery &q, uint32_t lanes, uint32_t *status, cudaStream_t s) {
    const uint64_t n = q.g.n;
    cudaError_t e = cudaMemsetAsync(q.vn, 0, sizeof(uint32_t) * 2 * n, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(q.qidx, 0xff, sizeof(uint32_t) * q.g.nnz, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(q.cross, 0, sizeof(uint32_t) * 2 * q.k, s);
    if (e == cudaSuccess && q.ret) e = cudaMemsetAsync(q.ret, 0, sizeof(uint32_t) * q.ret_cap, s);
    if (e != cudaSuccess) return cuda_fail(e, "shared batch setup");
    const uint32_t bouquet = 32u * lanes;
    count_launches(3);
    shared_prepare_kernel<<<blocks_for(q.k, kThreads), kThreads, 0, s>>>(q.g, q.uv, q.k, q.tau, q.nwalks, q.qinfo,
                                                                         q.vn, q.vt, q.qidx, status);
    vertex_tasks_kernel<<<blocks_for(n, kThreads), kThreads, 0, s>>>(n, q.vn, bouquet, q.tasks);
    int rc = scan_u32_to_u64_ws(q.tasks, q.vbegin, n, q.ws, q.ws_bytes, s);
    if (rc) return rc;
    build_bucket_kernel<<<blocks_for(n, kThreads), kThreads, 0, s>>>(q.vbegin, n, q.bucket);
    rc = scan_u32_to_u64_ws(q.vt, q.rbegin, n, q.ws, q.ws_bytes, s);
    if (rc) return rc;
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

template <int W, bool C>
int shared_batch_grid(int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shared_batch_count_kernel<W, C>, kThreads, 0));
    *grid = sms * (per_sm < 1 ? 1 : per_sm);
    return BQ_OK;
}

int shared_batch_create(const bq_aesc_query *queries, uint32_t n_queries, const Sampler &smp, SharedBatch **out,
                        uint64_t *edges) {
    *out = nullptr;
    int dev = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    SharedBatch *b = new (std::nothrow) SharedBatch();
    if (!b) return fail(BQ_ENOMEM, "host allocation failed");
    b->device = dev;
    b->smp = smp;
    b->lanes = shared_walks_per_lane(smp);
    b->q.resize(n_queries);
    int rc = status_word(dev, &b->status);
    uint32_t *plan_status = nullptr;  // the plan run at creation reports nothing to bq_sync
    if (rc == BQ_OK && cudaMalloc(&plan_status, sizeof(uint32_t)) != cudaSuccess)
        rc = fail(BQ_ENOMEM, "cannot allocate the batch buffers");
    if (rc == BQ_OK && cudaMemset(plan_status, 0, sizeof(uint32_t)) != cudaSuccess)
        rc = fail(BQ_ECUDA, "cudaMemset");
    std::vector<SharedQueryDesc> qd(n_queries);
    for (uint32_t i = 0; i < n_queries && rc == BQ_OK; ++i) {
        const bq_aesc_query &in = queries[i];
        const bq_graph *g = in.graph;
        SharedBatchQuery &q = b->q[i];
        if (!g) rc = fail(BQ_EINVAL, "query %u: graph is NULL", i);
        else if (g->device != dev) rc = fail(BQ_EINVAL, "query %u: graph lives on device %d, not %d", i, g->device, dev);
        else if (!g->d_rec8) rc = fail(BQ_EINVAL, "query %u: batches need graphs with nnz < 2^32", i);
        else if (in.k && (!in.tau_dev || !in.nwalks_dev || !in.counts_dev || !in.sc_dev))
            rc = fail(BQ_EINVAL, "query %u: tau, nwalks, counts or sc is NULL", i);
        else if (!in.edges_uv_dev && (in.k != g->nnz / 2 || in.k != g->m_upper))
            rc = fail(BQ_EINVAL, "query %u: all-edges query needs k = m = %llu", i, (unsigned long long)(g->nnz / 2));
        if (rc) break;
        q.g = g->view();
        q.seed = in.seed;
        q.k = in.k;
        q.uv = in.edges_uv_dev;
        q.tau = in.tau_dev;
        q.nwalks = in.nwalks_dev;
        q.counts = in.counts_dev;
        q.sc = in.sc_dev;
        b->edges += in.k;
        if (q.k == 0) continue;
        const uint64_t n = q.g.n;
        q.ws_bytes = scan_u32_to_u64_ws_bytes(n);
        const size_t b_qinfo = align16(sizeof(SharedQuery) * q.k), b_vnt = align16(sizeof(uint32_t) * 2 * n);
        const size_t b_tasks = align16(sizeof(uint32_t) * n);
        const size_t b_vbegin = align16(sizeof(uint64_t) * (n + 1) + sizeof(uint32_t) * bucket_count(n));
        const size_t b_rbegin = align16(sizeof(uint64_t) * (n + 1)), b_qidx = align16(sizeof(uint32_t) * q.g.nnz);
        const size_t b_cross = align16(sizeof(uint32_t) * 2 * q.k);
        const size_t bytes = b_qinfo + b_vnt + b_tasks + b_vbegin + b_rbegin + b_qidx + b_cross + align16(q.ws_bytes);
        if (cudaMalloc(&q.buf, bytes) != cudaSuccess ||
            (!q.uv && cudaMalloc(&q.own_uv, sizeof(uint32_t) * 2 * q.k) != cudaSuccess)) {
            rc = fail(BQ_ENOMEM, "query %u: cannot allocate %zu bytes of plan buffers", i, bytes);
            break;
        }
        char *p = q.buf;
        q.qinfo = (SharedQuery *)p;
        p += b_qinfo;
        q.vn = (uint32_t *)p;
        q.vt = q.vn + n;
        p += b_vnt;
        q.tasks = (uint32_t *)p;
        p += b_tasks;
        q.vbegin = (uint64_t *)p;
        q.bucket = (uint32_t *)(q.vbegin + n + 1);
        p += b_vbegin;
        q.rbegin = (uint64_t *)p;
        p += b_rbegin;
        q.qidx = (uint32_t *)p;
        p += b_qidx;
        q.cross = (uint32_t *)p;
        p += b_cross;
        q.ws = p;
        if (!q.uv) {  // the canonical edge list of an all-edges query is built once
            rc = launch_canonical_edges(q.g, q.own_uv, 0);
            q.uv = q.own_uv;
        }
        // one plan now sizes the return histograms: sum over vertices of tau_x
        if (rc == BQ_OK) rc = shared_plan(q, (uint32_t)b->lanes, plan_status, 0);
        uint64_t ret_len = 0;
        if (rc == BQ_OK && (cudaMemcpy(&ret_len, q.rbegin + n, sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess))
            rc = fail(BQ_ECUDA, "query %u: reading the plan", i);
        if (rc) break;
        q.ret_cap = ret_len + 1;
        if (cudaMalloc(&q.ret, sizeof(uint32_t) * q.ret_cap) != cudaSuccess) {
            rc = fail(BQ_ENOMEM, "query %u: cannot allocate its return histograms", i);
            break;
        }
        SharedQueryDesc &d = qd[i];
        d.g = graph_desc(g);
        d.seed = q.seed;
        d.n = n;
        d.vn = q.vn;
        d.vt = q.vt;
        d.vbegin = q.vbegin;
        d.bucket = q.bucket;
        d.rbegin = q.rbegin;
        d.qidx = q.qidx;
        d.qinfo = q.qinfo;
        d.ret = q.ret;
        d.cross = q.cross;
        d.ret_cap = q.ret_cap;
    }
    cudaFree(plan_status);
    if (rc == BQ_OK) {
        // a query without edges keeps a descriptor with no tasks: its vbegin
        // points at a zero word
        for (uint32_t i = 0; i < n_queries; ++i)
            if (b->q[i].k == 0) qd[i].n = 0;
        cudaError_t e = cudaMalloc(&b->d_qd, sizeof(SharedQueryDesc) * (n_queries ? n_queries : 1));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_qbase, sizeof(uint64_t) * (n_queries + 1));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned long long) * 2);
        if (e == cudaSuccess) e = cudaMemset(b->d_next, 0, sizeof(unsigned long long) * 2);
        for (uint32_t i = 0; i < n_queries && e == cudaSuccess; ++i)
            if (b->q[i].k == 0) qd[i].vbegin = reinterpret_cast<const uint64_t *>(b->d_next + 1);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_qd, qd.data(), sizeof(SharedQueryDesc) * n_queries, cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            rc = e == cudaErrorMemoryAllocation ? fail(BQ_ENOMEM, "cannot allocate the batch buffers")
                                                : cuda_fail(e, "shared batch create");
    }
    if (rc == BQ_OK) {
        rc = smp.kind == 1   ? shared_batch_grid<kSharedW, true>(&b->grid)
             : b->lanes == 4 ? shared_batch_grid<4, false>(&b->grid)
             : b->lanes == 8 ? shared_batch_grid<8, false>(&b->grid)
                             : shared_batch_grid<2, false>(&b->grid);
    }
    if (rc) {
        shared_batch_free_impl(b);
        return rc;
    }
    *out = b;
    *edges = b->edges;
    return BQ_OK;
}

int shared_batch_run(SharedBatch *b, cudaStream_t s) {
    const uint32_t nq = (uint32_t)b->q.size();
    BQ_CUDA(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s));
    {
        ProfScope prof(kProfAescAux, s);
        for (const SharedBatchQuery &q : b->q) {
            if (q.k == 0) continue;
            const int rc = shared_plan(q, (uint32_t)b->lanes, b->status, s);
            if (rc) return rc;
        }
        count_launches(1);
        shared_qbase_kernel<<<1, 32, 0, s>>>(b->d_qd, nq, b->d_qbase);
    }
    {
        ProfScope prof(kProfAesc, s);
        count_launches(1);
        const SharedQueryDesc *qd = b->d_qd;
        if (b->smp.kind == 1)
            shared_batch_count_kernel<kSharedW, true><<<b->grid, kThreads, 0, s>>>(qd, b->d_qbase, nq, b->smp, b->d_next);
        else if (b->lanes == 4)
            shared_batch_count_kernel<4, false><<<b->grid, kThreads, 0, s>>>(qd, b->d_qbase, nq, b->smp, b->d_next);
        else if (b->lanes == 8)
            shared_batch_count_kernel<8, false><<<b->grid, kThreads, 0, s>>>(qd, b->d_qbase, nq, b->smp, b->d_next);
        else
            shared_batch_count_kernel<2, false><<<b->grid, kThreads, 0, s>>>(qd, b->d_qbase, nq, b->smp, b->d_next);
        BQ_CUDA(cudaGetLastError());
    }
    ProfScope prof(kProfAescAux, s);
    for (const SharedBatchQuery &q : b->q) {
        if (q.k == 0) continue;
        count_launches(1);
        shared_finalize_kernel<<<blocks_for(q.k, kThreads), kThreads, 0, s>>>(
            q.qinfo, q.k, q.g.offsets, q.vn, q.rbegin, q.g.n, q.ret_cap, q.ret, q.cross, q.counts, nullptr, q.sc,
            b->status);
    }
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

void shared_batch_free(SharedBatch *b) { shared_batch_free_impl(b); }

}  // namespace bq

extern "C" {

int bq_aesc_estimate_shared(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev, uint64_t k,
                            const uint32_t *tau_dev, const uint32_t *nwalks_dev, const bq_sampler *sampler,
                            uint32_t flags, uint32_t *counts_dev, uint32_t *nused_dev, double *sc_dev, void *stream) {
    using namespace bq;
    NvtxRange nvtx_range("bq_aesc_estimate_shared");
    clear_error();
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (flags & ~BQ_HOST_IO) return fail(BQ_EINVAL, "unknown AESC flags 0x%x", flags);
    if (k && (!tau_dev || !nwalks_dev || !counts_dev || !sc_dev))
        return fail(BQ_EINVAL, "tau, nwalks, counts or sc is NULL");
    if (!edges_uv_dev && (k != g->nnz / 2 || k != g->m_upper))
        return fail(BQ_EINVAL, "all-edges estimate needs k = m = %llu (got %llu; %llu edges above the diagonal)",
                    (unsigned long long)(g->nnz / 2), (unsigned long long)k, (unsigned long long)g->m_upper);
    Sampler smp;
    int rc = validate_sampler(sampler, smp);
    if (rc) return rc;
    if (k == 0) return BQ_OK;
    DeviceGuard guard(g->device);
    uint32_t *status = nullptr;
    rc = status_word(g->device, &status);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!(flags & BQ_HOST_IO))
        return launch_aesc_shared(g->view(), seed, edges_uv_dev, k, tau_dev, nwalks_dev, smp, counts_dev, nused_dev,
                                  sc_dev, status, s);

    const size_t eb = edges_uv_dev ? sizeof(uint32_t) * 2 * k : 0;
    const size_t tb = sizeof(uint32_t) * k, cb = sizeof(uint32_t) * 4 * k, scb = sizeof(double) * k;
    char *buf = nullptr;
    rc = scratch_alloc((void **)&buf, scb + cb + 4 * tb + eb, s);
    if (rc) return rc;
    double *d_sc = (double *)buf;
    uint32_t *d_counts = (uint32_t *)(buf + scb);
    uint32_t *d_tau = (uint32_t *)(buf + scb + cb);
    uint32_t *d_nw = (uint32_t *)(buf + scb + cb + tb);
    uint32_t *d_nused = (uint32_t *)(buf + scb + cb + 2 * tb);
    uint32_t *d_uv = edges_uv_dev ? (uint32_t *)(buf + scb + cb + 4 * tb) : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_tau, tau_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_nw, nwalks_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d_uv) e = cudaMemcpyAsync(d_uv, edges_uv_dev, eb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "host-io upload");
    if (rc == BQ_OK)
        rc = launch_aesc_shared(g->view(), seed, d_uv, k, d_tau, d_nw, smp, d_counts, d_nused, d_sc, status, s);
    if (rc == BQ_OK) {
        e = cudaMemcpyAsync(counts_dev, d_counts, cb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc_dev, d_sc, scb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && nused_dev)
            e = cudaMemcpyAsync(nused_dev, d_nused, 2 * tb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "host-io download");
    }
    scratch_free(buf, s);
    if (rc == BQ_OK) rc = bq_sync(stream);
    else cudaStreamSynchronize(s);
    return rc;
}

}  // extern "C"
