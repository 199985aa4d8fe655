// Graph store: validation of a device CSR, per-vertex records, canonical
// edge numbering, and the device-wide exclusive scan used across the library.
//
// The adjacency Gamma(v) and degree d(v) are the notation of Sec. 2 (Table of
// notation); Alg. 2 and Alg. 3 index Gamma(cur)[k], so every step needs the
// row start and the row length of the current vertex.  They are packed into
// one aligned record per vertex so that a step reads them with one load.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace bq {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

// ------------------------------------------------------------------ scan

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if ((threadIdx.x & 31) >= (unsigned)d) x += y;
    }
    return x;
}

// Exclusive scan of one block tile held as kScanItems values per thread
// (blocked arrangement); `total` receives the tile sum in every thread.
template <typename Out>
__device__ void block_exclusive_scan(Out (&v)[kScanItems], Out &total) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ Out warp_sums[kWarps];
    __shared__ Out tile_total;
    Out local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) local += v[i];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const Out incl = warp_inclusive_scan(local);
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const Out ws = lane < kWarps ? warp_sums[lane] : (Out)0;
        const Out wi = warp_inclusive_scan(ws);
        if (lane < kWarps) warp_sums[lane] = wi - ws;
        if (lane == kWarps - 1) tile_total = wi;
    }
    __syncthreads();
    Out run = warp_sums[wid] + incl - local;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const Out x = v[i];
        v[i] = run;
        run += x;
    }
    total = tile_total;
}

template <typename In, typename Out>
__global__ void tile_reduce_kernel(const In *__restrict__ in, uint64_t n, Out *__restrict__ sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    Out local = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) local += (Out)in[idx];
    }
    __shared__ Out warp_sums[kScanThreads / 32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) local += __shfl_down_sync(0xffffffffu, local, d);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        Out t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += warp_sums[w];
        sums[blockIdx.x] = t;
    }
}

// out[i] = offsets[block] + exclusive prefix within the tile; the last tile
// also writes out[n] = grand total.
template <typename In, typename Out>
__global__ void tile_scan_kernel(const In *__restrict__ in, uint64_t n,
                                 const Out *__restrict__ tile_offsets, Out *__restrict__ out) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    Out v[kScanItems];
    // blocked arrangement: thread t owns items base + t*kScanItems + i
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t idx = base + (uint64_t)threadIdx.x * kScanItems + i;
        v[i] = idx < n ? (Out)in[idx] : (Out)0;
    }
    Out total;
    block_exclusive_scan<Out>(v, total);
    const Out off = tile_offsets ? tile_offsets[blockIdx.x] : (Out)0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const uint64_t idx = base + (uint64_t)threadIdx.x * kScanItems + i;
        if (idx < n) out[idx] = off + v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = off + total;
}

template <typename In, typename Out>
int scan_impl(const In *in, Out *out, uint64_t n, cudaStream_t s) {
    if (n == 0) {
        BQ_CUDA(cudaMemsetAsync(out, 0, sizeof(Out), s));
        return BQ_OK;
    }
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        count_launches(1);
        tile_scan_kernel<In, Out><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        BQ_CUDA(cudaGetLastError());
        return BQ_OK;
    }
    Out *sums = nullptr;
    int rc = scratch_alloc((void **)&sums, sizeof(Out) * (2 * tiles + 1), s);
    if (rc) return rc;
    Out *sum_prefix = sums + tiles;
    count_launches(2);
    tile_reduce_kernel<In, Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    rc = scan_impl<Out, Out>(sums, sum_prefix, tiles, s);
    if (rc == BQ_OK) {
        tile_scan_kernel<In, Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sum_prefix, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "tile_scan_kernel");
    }
    scratch_free(sums, s);
    return rc;
}

// Workspace bytes scan_ws_impl needs for n items (tile sums and their prefix
// at every level of the recursion).
template <typename Out>
size_t scan_ws_bytes_impl(uint64_t n) {
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles <= 1) return 0;
    const size_t here = (sizeof(Out) * (2 * tiles + 1) + 255) & ~(size_t)255;
    return here + scan_ws_bytes_impl<Out>(tiles);
}

// The same scan as scan_impl, with its temporary tile sums taken from a
// caller-provided workspace instead of the stream-ordered pool.
template <typename In, typename Out>
int scan_ws_impl(const In *in, Out *out, uint64_t n, char *ws, size_t ws_bytes, cudaStream_t s) {
    if (n == 0) {
        BQ_CUDA(cudaMemsetAsync(out, 0, sizeof(Out), s));
        return BQ_OK;
    }
    const uint64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        count_launches(1);
        tile_scan_kernel<In, Out><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        BQ_CUDA(cudaGetLastError());
        return BQ_OK;
    }
    const size_t here = (sizeof(Out) * (2 * tiles + 1) + 255) & ~(size_t)255;
    if (ws_bytes < here) return fail(BQ_EINVAL, "scan workspace too small");
    Out *sums = (Out *)ws;
    Out *sum_prefix = sums + tiles;
    count_launches(2);
    tile_reduce_kernel<In, Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
    int rc = scan_ws_impl<Out, Out>(sums, sum_prefix, tiles, ws + here, ws_bytes - here, s);
    if (rc) return rc;
    tile_scan_kernel<In, Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sum_prefix, out);
    BQ_CUDA(cudaGetLastError());
    return BQ_OK;
}

// ------------------------------------------------------------ validation

struct CheckResult {
    unsigned long long bad_offset;  // first v with offsets[v] > offsets[v+1]
    unsigned long long bad_id;      // first v whose row holds an id >= n
    unsigned long long self_loop;   // first v whose row holds v
    unsigned long long unsorted;    // first v whose row is not strictly increasing
    unsigned long long asymmetric;  // first v with u in row v but v not in row u
    unsigned int min_deg;
    unsigned int max_deg;
};

__global__ void check_offsets_kernel(const int64_t *__restrict__ off, uint32_t n, CheckResult *res) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        if (off[v] > off[v + 1]) atomicMin(&res->bad_offset, (unsigned long long)v);
    }
}

// One warp per vertex: bounds, self-loops, sortedness, degree range and the
// number of neighbours above v (canonical edge numbering).
__global__ void check_rows_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ nbrs,
                                  uint32_t n, CheckResult *res, uint32_t *__restrict__ upper) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nwarps) {
        const int64_t lo = off[v], hi = off[v + 1];
        bool bad_id = false, self = false, unsorted = false;
        uint32_t above = 0;
        for (int64_t j = lo + lane; j < hi; j += 32) {
            const uint32_t x = nbrs[j];
            bad_id |= x >= n;
            self |= x == (uint32_t)v;
            unsorted |= (j > lo) && (nbrs[j - 1] >= x);
            above += x > (uint32_t)v;
        }
        bad_id = __any_sync(0xffffffffu, bad_id);
        self = __any_sync(0xffffffffu, self);
        unsorted = __any_sync(0xffffffffu, unsorted);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) above += __shfl_down_sync(0xffffffffu, above, d);
        if (lane == 0) {
            if (bad_id) atomicMin(&res->bad_id, (unsigned long long)v);
            if (self) atomicMin(&res->self_loop, (unsigned long long)v);
            if (unsorted) atomicMin(&res->unsorted, (unsigned long long)v);
            const unsigned int deg = (unsigned int)(hi - lo);
            atomicMin(&res->min_deg, deg);
            atomicMax(&res->max_deg, deg);
            upper[v] = above;
        }
    }
}

__device__ __forceinline__ bool row_contains(const uint32_t *__restrict__ nbrs, int64_t lo,
                                             int64_t hi, uint32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        const uint32_t x = nbrs[mid];
        if (x == key) return true;
        if (x < key) lo = mid + 1;
        else hi = mid;
    }
    return false;
}

// Needs rows sorted and ids in range (checked before it runs).
__global__ void check_symmetry_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ nbrs,
                                      uint32_t n, CheckResult *res) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp; v < n; v += nwarps) {
        bool asym = false;
        for (int64_t j = off[v] + lane; j < off[v + 1]; j += 32) {
            const uint32_t x = nbrs[j];
            asym |= !row_contains(nbrs, off[x], off[x + 1], (uint32_t)v);
        }
        if (__any_sync(0xffffffffu, asym) && lane == 0)
            atomicMin(&res->asymmetric, (unsigned long long)v);
    }
}

__global__ void build_records_kernel(const int64_t *__restrict__ off, uint32_t n, uint2 *rec8,
                                     uint4 *rec16) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t lo = off[v];
        const uint32_t deg = (uint32_t)(off[v + 1] - lo);
        if (rec8) rec8[v] = make_uint2((uint32_t)lo, deg);
        else rec16[v] = make_uint4((uint32_t)lo, (uint32_t)((uint64_t)lo >> 32), deg, 0u);
    }
}

// Edge record of CSR entry j: the neighbour's id, row offset and degree.
__global__ void build_edges_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ nbrs,
                                   uint64_t nnz, uint32_t sh_off, uint32_t sh_deg, uint64_t *edge8,
                                   uint4 *edge16) {
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < nnz;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x = nbrs[j];
        const uint64_t lo = (uint64_t)off[x];
        const uint64_t deg = (uint64_t)off[x + 1] - lo;
        if (edge8) edge8[j] = (uint64_t)x | (lo << sh_off) | (deg << sh_deg);
        else edge16[j] = make_uint4(x, (uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)deg);
    }
}

// Chunk c of the packed ids holds entries c*q .. c*q + q - 1, entry i of the
// chunk at bits [i*bits, (i+1)*bits) of the 128-bit chunk (word 0 = bits
// 0..31).
__global__ void build_packed_ids_kernel(const uint32_t *__restrict__ nbrs, uint64_t nnz, uint32_t bits, uint32_t q,
                                        uint64_t chunks, uint4 *__restrict__ pk) {
    for (uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c < chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        for (uint32_t i = 0; i < q; ++i) {
            const uint64_t j = c * q + i;
            if (j >= nnz) break;
            const uint64_t v = nbrs[j];
            const uint32_t bit = i * bits;
            const uint32_t wi = bit >> 5, sh = bit & 31;
            w[wi] |= (uint32_t)(v << sh);
            if (sh + bits > 32) w[wi + 1] |= (uint32_t)(v >> (32 - sh));
        }
        pk[c] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Degree-relabelled copy: the entries of internal row x (original vertex
// orig[x]) as internal ids, in the original order, at the row's new place.
// One warp per row.
__global__ void relabel_rows_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ nbrs,
                                    const uint32_t *__restrict__ orig, const uint32_t *__restrict__ new_of,
                                    const int64_t *__restrict__ off_new, uint32_t n, uint32_t *__restrict__ out) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t x = warp; x < n; x += nwarps) {
        const uint32_t v = orig[x];
        const int64_t lo = off[v], d = off[v + 1] - lo, dst = off_new[x];
        for (int64_t i = lane; i < d; i += 32) out[dst + i] = new_of[nbrs[lo + i]];
    }
}

// rec8[x] = original id | row offset << sh_off | degree << sh_deg of
// internal vertex x; a degree that needs more than deg_bits bits (only the
// first internal ids, which the kernels serve from shared memory) is stored
// as 0.
__global__ void relabel_rec8_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ orig,
                                    const int64_t *__restrict__ off_new, uint32_t n, uint32_t deg_bits,
                                    uint32_t sh_off, uint32_t sh_deg, uint64_t *__restrict__ rec8) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = orig[x];
        uint64_t d = (uint64_t)(off[v + 1] - off[v]);
        if ((d >> deg_bits) != 0) d = 0;
        rec8[x] = (uint64_t)v | ((uint64_t)off_new[x] << sh_off) | (d << sh_deg);
    }
}

// rec[x] = {row offset, degree, original id, 0} of internal vertex x.
__global__ void relabel_records_kernel(const int64_t *__restrict__ off, const uint32_t *__restrict__ orig,
                                       const int64_t *__restrict__ off_new, uint32_t n, uint4 *__restrict__ rec) {
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = orig[x];
        rec[x] = make_uint4((uint32_t)off_new[x], (uint32_t)(off[v + 1] - off[v]), v, 0u);
    }
}

// Hub table: every vertex with a neighbour bids for slot hash(v); the highest
// degree wins (ties: the smaller id).  key = degree << 32 | (2^32 - 1 - v).
__global__ void hub_select_kernel(const int64_t *__restrict__ off, uint32_t n, uint32_t slots,
                                  unsigned long long *__restrict__ best) {
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t deg = (uint64_t)(off[v + 1] - off[v]);
        if (deg == 0) continue;
        const uint32_t slot = hub_slot((uint32_t)v, slots);
        atomicMax(best + slot, (unsigned long long)((deg << 32) | (0xffffffffull - v)));
    }
}

__global__ void hub_finish_kernel(const unsigned long long *__restrict__ best, uint32_t slots,
                                  uint32_t *__restrict__ tag) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x)
        tag[i] = best[i] ? 0xffffffffu - (uint32_t)best[i] : kNoHub;
}

uint32_t bits_for(uint64_t max_value) {
    uint32_t b = 1;
    while (b < 64 && (max_value >> b) != 0) ++b;
    return b;
}

unsigned grid_for(uint64_t items, int threads, int per_thread = 1) {
    uint64_t blocks = (items + (uint64_t)threads * per_thread - 1) / ((uint64_t)threads * per_thread);
    if (blocks < 1) blocks = 1;
    if (blocks > 65535ull * 32) blocks = 65535ull * 32;
    return (unsigned)blocks;
}

}  // namespace

int scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s) {
    return scan_impl<uint32_t, uint64_t>(in, out, n, s);
}

int scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, s);
}

size_t scan_u32_ws_bytes(uint64_t n) { return scan_ws_bytes_impl<uint32_t>(n); }

size_t scan_u32_to_u64_ws_bytes(uint64_t n) { return scan_ws_bytes_impl<uint64_t>(n); }

int scan_u32_to_u64_ws(const uint32_t *in, uint64_t *out, uint64_t n, void *ws, size_t ws_bytes, cudaStream_t s) {
    return scan_ws_impl<uint32_t, uint64_t>(in, out, n, (char *)ws, ws_bytes, s);
}

int scan_u32_ws(const uint32_t *in, uint32_t *out, uint64_t n, void *ws, size_t ws_bytes, cudaStream_t s) {
    return scan_ws_impl<uint32_t, uint32_t>(in, out, n, (char *)ws, ws_bytes, s);
}

// The degree-relabelled copy of a packed-id graph (bq_tuning.hub_relabel):
// internal ids follow (degree desc, original id asc), vertices without
// neighbours last, so every prefix 0..H-1 holds the H highest-degree
// vertices.  The walk kernels serve such a prefix from shared memory: the
// plain relabel kernel the first rl_hubs (as many 12-byte entries as
// hub_slots * 16 bytes of shared memory hold), the 8-byte-hub kernel as many
// 8-byte entries as fit in the same bytes, at least rl_fit (the vertices
// whose degree does not fit the records' degree field).  The degree order
// also puts the records of the most visited non-hubs side by side (8.54
// against 8.83 ms per R-MAT 20 batch for the plain relabel kernel, against
// the earlier order by original id).
int build_relabelled(bq_graph *g, uint32_t bits, uint32_t q, uint64_t chunks, cudaStream_t s) {
    const uint32_t n = g->n;
    std::vector<int64_t> off(n + 1);
    BQ_CUDA(cudaMemcpy(off.data(), g->d_offsets, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost));
    auto deg = [&](uint32_t v) { return off[v + 1] - off[v]; };
    // internal order: degree descending, ids ascending within a degree (a
    // stable counting sort over the degrees, linear in n + max degree)
    int64_t max_deg = 0;
    for (uint32_t v = 0; v < n; ++v) max_deg = std::max(max_deg, deg(v));
    std::vector<uint64_t> first((size_t)max_deg + 1, 0);
    for (uint32_t v = 0; v < n; ++v) ++first[(size_t)deg(v)];
    uint64_t pos = 0;
    for (int64_t d = max_deg; d >= 0; --d) {
        const uint64_t c = first[(size_t)d];
        first[(size_t)d] = pos;
        pos += c;
    }
    std::vector<uint32_t> orig(n);
    for (uint32_t v = 0; v < n; ++v) orig[first[(size_t)deg(v)]++] = v;
    uint32_t live = 0;
    while (live < n && deg(orig[live]) > 0) ++live;
    const uint64_t cap = ((uint64_t)tuning_hub_slots() * 16 - 4) / 12;
    const uint32_t hubs = (uint32_t)std::min<uint64_t>(cap, live);
    if (hubs == 0) return BQ_OK;
    std::vector<uint32_t> new_of(n);
    for (uint32_t x = 0; x < n; ++x) new_of[orig[x]] = x;
    std::vector<int64_t> off_new(n + 1);
    off_new[0] = 0;
    for (uint32_t x = 0; x < n; ++x) off_new[x + 1] = off_new[x] + deg(orig[x]);
    // 8-byte records when id, offset and the largest non-hub degree fit
    const int64_t max_other = hubs < n ? deg(orig[hubs]) : 0;
    const uint32_t b_id = bits_for(n > 0 ? n - 1 : 0), b_off = bits_for(g->nnz), b_deg = bits_for(max_other);
    if (b_id + b_off + b_deg > 64) return BQ_OK;  // no relabelled copy
    uint32_t fit = 0;  // first internal id whose degree fits b_deg bits
    while (fit < n && (deg(orig[fit]) >> b_deg) != 0) ++fit;
    uint32_t *d_orig = nullptr, *d_tmp = nullptr;
    int64_t *d_off_new = nullptr;
    cudaError_t e = cudaMalloc(&g->d_rl_new, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_rl_rec, sizeof(uint4) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_rl_rec8, sizeof(uint64_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_rl_pk, sizeof(uint4) * chunks);
    if (e == cudaSuccess) e = cudaMalloc(&d_orig, sizeof(uint32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_off_new, sizeof(int64_t) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_tmp, sizeof(uint32_t) * g->nnz);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_rl_new, new_of.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_orig, orig.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(d_off_new, off_new.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        relabel_rows_kernel<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(g->d_offsets, g->d_nbrs, d_orig,
                                                                           g->d_rl_new, d_off_new, n, d_tmp);
        build_packed_ids_kernel<<<grid_for(chunks, 256), 256, 0, s>>>(d_tmp, g->nnz, bits, q, chunks, g->d_rl_pk);
        relabel_records_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->d_offsets, d_orig, d_off_new, n, g->d_rl_rec);
        relabel_rec8_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->d_offsets, d_orig, d_off_new, n, b_deg, b_id,
                                                             b_id + b_off, g->d_rl_rec8);
        e = cudaStreamSynchronize(s);
    }
    cudaFree(d_orig);
    cudaFree(d_off_new);
    cudaFree(d_tmp);
    if (e != cudaSuccess) return cuda_fail(e, "degree-relabelled copy");
    g->rl_hubs = hubs;
    g->rl_sh_off = b_id;
    g->rl_sh_deg = b_id + b_off;
    g->rl_mask_id = b_id >= 32 ? 0xffffffffu : ((1u << b_id) - 1u);
    g->rl_mask_off = b_off >= 64 ? ~0ull : ((1ull << b_off) - 1ull);
    g->rl_bits_deg = b_deg;
    g->rl_live = live;
    g->rl_fit = fit;
    g->device_bytes += sizeof(uint32_t) * n + sizeof(uint4) * n + sizeof(uint64_t) * n + sizeof(uint4) * chunks;
    return BQ_OK;
}

int graph_build(bq_graph *g, uint32_t flags, cudaStream_t s) {
    const uint32_t n = g->n;
    // offsets[0] and offsets[n] against nnz
    int64_t ends[2] = {0, 0};
    BQ_CUDA(cudaMemcpyAsync(&ends[0], g->d_offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BQ_CUDA(cudaMemcpyAsync(&ends[1], g->d_offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BQ_CUDA(cudaStreamSynchronize(s));
    if (ends[0] != 0) return fail(BQ_EGRAPH, "offsets[0] = %lld, expected 0", (long long)ends[0]);
    if (ends[1] < 0 || (uint64_t)ends[1] != g->nnz)
        return fail(BQ_EGRAPH, "offsets[n] = %lld does not match nnz = %llu", (long long)ends[1],
                    (unsigned long long)g->nnz);
    if (g->nnz % 2 != 0) return fail(BQ_EGRAPH, "nnz = %llu is odd: an undirected CSR stores each edge twice",
                                     (unsigned long long)g->nnz);

    CheckResult *res = nullptr;
    uint32_t *upper = nullptr;
    BQ_CUDA(cudaMalloc(&res, sizeof(CheckResult)));
    CheckResult init;
    init.bad_offset = init.bad_id = init.self_loop = init.unsorted = init.asymmetric = ~0ull;
    init.min_deg = 0xffffffffu;
    init.max_deg = 0;
    int rc = BQ_OK;
    CheckResult h;
    cudaError_t e = cudaMemcpyAsync(res, &init, sizeof(init), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMalloc(&upper, sizeof(uint32_t) * ((size_t)n + 1));
    if (e != cudaSuccess) {
        cudaFree(res);
        return cuda_fail(e, "graph validation setup");
    }
    if (n > 0) {
        check_offsets_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->d_offsets, n, res);
        e = cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "check_offsets_kernel");
            goto done;
        }
        if (h.bad_offset != ~0ull) {
            rc = fail(BQ_EGRAPH, "offsets decrease at vertex %llu", h.bad_offset);
            goto done;
        }
        check_rows_kernel<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(g->d_offsets, g->d_nbrs, n, res,
                                                                           upper);
        e = cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "check_rows_kernel");
            goto done;
        }
        if (h.bad_id != ~0ull) {
            rc = fail(BQ_EGRAPH, "row %llu holds a vertex id >= n = %u", h.bad_id, n);
            goto done;
        }
        if (h.self_loop != ~0ull) {
            rc = fail(BQ_EGRAPH, "vertex %llu has a self-loop", h.self_loop);
            goto done;
        }
        if (!(flags & BQ_SKIP_VALIDATE)) {
            if (h.unsorted != ~0ull) {
                rc = fail(BQ_EGRAPH, "row %llu is not strictly increasing (unsorted or duplicate entry)",
                          h.unsorted);
                goto done;
            }
            check_symmetry_kernel<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(g->d_offsets, g->d_nbrs,
                                                                                   n, res);
            e = cudaMemcpyAsync(&h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "check_symmetry_kernel");
                goto done;
            }
            if (h.asymmetric != ~0ull) {
                rc = fail(BQ_EGRAPH, "row %llu lists a neighbour whose row does not list it (asymmetric)",
                          h.asymmetric);
                goto done;
            }
        }
        g->min_degree = h.min_deg;
        g->max_degree = h.max_deg;
    }
    // records
    {
        const int layout = tuning_layout();
        const bool compact = g->nnz < (1ull << 32) && layout != 4;
        size_t rec_bytes = (size_t)n * (compact ? sizeof(uint2) : sizeof(uint4));
        void *rec = nullptr;
        e = cudaMalloc(&rec, rec_bytes > 0 ? rec_bytes : 16);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc(records)");
            goto done;
        }
        if (compact) g->d_rec8 = (uint2 *)rec;
        else g->d_rec16 = (uint4 *)rec;
        g->device_bytes += rec_bytes;
        if (n > 0)
            build_records_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->d_offsets, n, g->d_rec8, g->d_rec16);
        e = cudaMalloc(&g->d_upper_before, sizeof(uint64_t) * ((size_t)n + 1));
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "cudaMalloc(upper_before)");
            goto done;
        }
        g->device_bytes += sizeof(uint64_t) * ((size_t)n + 1);
        rc = scan_u32_to_u64(upper, g->d_upper_before, n, s);
        if (rc) goto done;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "graph_build");
            goto done;
        }
        uint64_t m_upper = 0;
        e = cudaMemcpy(&m_upper, g->d_upper_before + n, sizeof(uint64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "graph_build readback");
            goto done;
        }
        g->m_upper = m_upper;
        if (!(flags & BQ_SKIP_VALIDATE) && 2 * m_upper != g->nnz) {
            rc = fail(BQ_EGRAPH, "edge count mismatch: %llu entries above the diagonal, nnz %llu",
                      (unsigned long long)m_upper, (unsigned long long)g->nnz);
            goto done;
        }
        // Automatic layout: when the 8-byte edge records fit in L2, a step is
        // one cached load (one L1 request instead of two: measured 1.5-1.7x
        // faster AESC on power-law graphs of 43 and 86 MB of records);
        // otherwise the smallest array a step reads at random (bit-packed
        // ids) keeps the most of it in L2 (faster at 173 MB, and for the
        // walk batch on R-MAT scale 20).
        int use = layout;
        if (layout == 1) {
            int dev = 0, l2 = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) l2 = 0;
            const bool fits = bits_for(n > 0 ? n - 1 : 0) + bits_for(g->nnz) + bits_for(g->max_degree) <= 64;
            use = (compact && fits && (g->nnz + n) * 8ull <= (uint64_t)l2) ? 2 : 5;
        }
        if (g->nnz > 0 && use == 5 && compact) {
            const uint32_t bits = bits_for(n > 0 ? n - 1 : 0);
            const uint32_t q = 128 / bits;
            if (q > 4) {  // fewer than 32 bits per id: packing saves memory
                const uint64_t chunks = (g->nnz + q - 1) / q;
                const size_t bytes = sizeof(uint4) * chunks;
                e = cudaMalloc(&g->d_pk, bytes);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "cudaMalloc(packed ids)");
                    goto done;
                }
                g->device_bytes += bytes;
                g->pk_bits = bits;
                g->pk_q = q;
                g->pk_mask = bits >= 32 ? 0xffffffffu : ((1u << bits) - 1u);
                build_packed_ids_kernel<<<grid_for(chunks, 256), 256, 0, s>>>(g->d_nbrs, g->nnz, bits, q, chunks,
                                                                              g->d_pk);
                e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "build_packed_ids_kernel");
                    goto done;
                }
                if (tuning_hub_relabel() && tuning_hub_slots() > 0) {
                    rc = build_relabelled(g, bits, q, chunks, s);
                    if (rc) goto done;
                }
            }
        }
        if (g->nnz > 0 && (use == 2 || use == 3)) {
            const uint32_t b_id = bits_for(n > 0 ? n - 1 : 0);
            const uint32_t b_off = bits_for(g->nnz);
            const uint32_t b_deg = bits_for(g->max_degree);
            const bool packed = use == 2 && b_id + b_off + b_deg <= 64;
            const size_t bytes = g->nnz * (packed ? sizeof(uint64_t) : sizeof(uint4));
            void *edges = nullptr;
            e = cudaMalloc(&edges, bytes);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "cudaMalloc(edge records)");
                goto done;
            }
            g->device_bytes += bytes;
            if (packed) {
                g->d_edge8 = (uint64_t *)edges;
                g->sh_off = b_id;
                g->sh_deg = b_id + b_off;
                g->mask_id = b_id >= 32 ? 0xffffffffu : ((1u << b_id) - 1u);
                g->mask_off = (b_off >= 64) ? ~0ull : ((1ull << b_off) - 1ull);
            } else {
                g->d_edge16 = (uint4 *)edges;
            }
            build_edges_kernel<<<grid_for(g->nnz, 256, 4), 256, 0, s>>>(g->d_offsets, g->d_nbrs, g->nnz, g->sh_off,
                                                                        g->sh_deg, g->d_edge8, g->d_edge16);
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "build_edges_kernel");
                goto done;
            }
        }
        g->layout = g->d_pk ? 5 : (g->d_edge8 ? 2 : (g->d_edge16 ? 3 : (compact ? 0 : 4)));
        const uint32_t cluster = (uint32_t)tuning_hub_cluster() > 1 ? (uint32_t)tuning_hub_cluster() : 1u;
        const uint32_t slots = (uint32_t)tuning_hub_slots() * cluster;
        if (slots > 0 && compact && n > 0) {
            unsigned long long *best = nullptr;
            e = cudaMalloc(&best, sizeof(unsigned long long) * slots);
            if (e == cudaSuccess) e = cudaMalloc(&g->d_hub_tag, sizeof(uint32_t) * slots);
            if (e == cudaSuccess) e = cudaMemsetAsync(best, 0, sizeof(unsigned long long) * slots, s);
            if (e == cudaSuccess) {
                hub_select_kernel<<<grid_for(n, 256), 256, 0, s>>>(g->d_offsets, n, slots, best);
                hub_finish_kernel<<<grid_for(slots, 256), 256, 0, s>>>(best, slots, g->d_hub_tag);
                e = cudaStreamSynchronize(s);
            }
            cudaFree(best);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "hub table");
                goto done;
            }
            g->hub_slots = slots;
            g->hub_cluster = cluster;
            g->device_bytes += sizeof(uint32_t) * slots;
        }
    }
done:
    cudaFree(res);
    cudaFree(upper);
    return rc;
}

int graph_fetch_host(bq_graph *g) {
    if (!g->h_offsets.empty()) return BQ_OK;
    int prev = 0;
    BQ_CUDA(cudaGetDevice(&prev));
    BQ_CUDA(cudaSetDevice(g->device));
    std::vector<int64_t> off((size_t)g->n + 1);
    std::vector<uint32_t> nb((size_t)g->nnz);
    cudaError_t e = cudaMemcpy(off.data(), g->d_offsets, sizeof(int64_t) * off.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && g->nnz)
        e = cudaMemcpy(nb.data(), g->d_nbrs, sizeof(uint32_t) * nb.size(), cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e, "graph_fetch_host");
    g->h_offsets.swap(off);
    g->h_nbrs.swap(nb);
    return BQ_OK;
}

}  // namespace bq
