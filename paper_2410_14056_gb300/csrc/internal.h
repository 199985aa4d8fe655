// Internal declarations shared by the translation units of libbouquet.
// Host-side only types plus the launch wrappers each .cu file exports.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <nvtx3/nvToolsExt.h>

#include "../../include/bouquet.h"

namespace bq {

// Bits of the per-device status word written by kernels (atomicOr).
enum StatusBits : uint32_t {
    kStatusBadStart = 1u << 0,   // walk start id >= n
    kStatusNoEdge = 1u << 1,     // AESC pair is not an edge
    kStatusOverflow = 1u << 2,   // a uint32 counter wrapped / plan too large
    kStatusBadIndex = 1u << 3,   // (checked builds) index out of range
    kStatusTimeout = 1u << 4,    // a bounded wait gave up
    kStatusRepeated = 1u << 5,   // an edge repeated among vertex-centric queries
    kStatusPlanGrew = 1u << 6,   // a shared batch's plan outgrew its histograms
};

constexpr uint32_t kNoHub = 0xffffffffu;
constexpr uint32_t kHubHash = 0x9E3779B1u;
constexpr uint32_t kHubSlotsMax = 13312;  // 16 B per slot: 208 KiB of shared memory
constexpr uint32_t kHub8Max = 28000;  // 8 B per hub: at most 219 KiB of shared memory

// Hub-table slot of vertex v: the high half of (v * kHubHash mod 2^32) * slots.
__host__ __device__ __forceinline__ uint32_t hub_slot(uint32_t v, uint32_t slots) {
    return (uint32_t)(((uint64_t)(v * kHubHash) * slots) >> 32);
}

// Stream reserved for walk-batch walks; AESC walks use stream 2 * edge + side.
constexpr uint64_t kBatchStream = 0x4000000000000000ull;
// Top bit of the stream selects the shared key of the coupled sampler.
constexpr uint64_t kGroupBit = 0x8000000000000000ull;

struct Sampler {
    uint32_t kind;   // 0 independent, 1 coupled (also the literal SABA word)
    uint32_t t;      // coupled: shared top bits; kSabaT: the literal SABA word
    uint32_t width;  // coupled: group width
};

// Sampler::t of the paper's SABA word taken literally (BQ_SAMPLER_SABA).
constexpr uint32_t kSabaT = 0xffffffffu;

// Device view of a graph.  Vertex records are 8 bytes {row offset, degree}
// when nnz < 2^32 (compact), else 16 bytes {offset lo, offset hi, degree, 0}.
struct DeviceGraph {
    uint32_t n;
    uint64_t nnz;
    const int64_t *offsets;  // n + 1
    const uint32_t *nbrs;    // nnz
    const uint2 *rec8;       // n, compact records (or null)
    const uint4 *rec16;      // n, wide records (or null)
    const uint64_t *upper_before;  // n + 1: edges {x,y}, x<y, with x < u
    // Edge records: entry j of the CSR carries everything the next step
    // needs about its neighbour x = nbrs[j]: {x, row offset of x, degree of
    // x}.  Packed into 64 bits (id | offset << sh_off | degree << sh_deg)
    // when the three fields fit, else 16 bytes {x, offset lo, offset hi,
    // degree}; null when the graph was built without them.
    const uint64_t *edge8;
    const uint4 *edge16;
    uint32_t sh_off, sh_deg;
    uint32_t mask_id;
    uint64_t mask_off;
    // Packed neighbour ids: `pk_q` ids of `pk_bits` bits per 16-byte chunk
    // (id i of chunk c at bits [i*pk_bits, (i+1)*pk_bits)), so that an id
    // never straddles a chunk and one aligned vector load reads it.
    const uint4 *pk;
    uint32_t pk_bits, pk_q, pk_mask;
    // Hub table: slot hub_slot(v, hub_slots) holds the highest-degree
    // vertex hashing there (kNoHub when empty); null if none.
    const uint32_t *hub_tag;
    uint32_t hub_slots;    // slots in all (hub_slot over this count)
    uint32_t hub_cluster;  // CTAs sharing the table (1: one CTA holds it)
    // Degree-relabelled copy for the walk batch (null if not built): internal
    // ids follow (degree desc, original id asc), vertices without neighbours
    // last, so internal ids x < H are the H highest-degree vertices for any
    // H; rows keep the original neighbour order.  rl_new[v] = internal id of
    // original v; rl_rec[x] = {row offset, degree, original id, 0}; rl_pk =
    // the rows' internal ids packed as `pk`.
    const uint4 *rl_pk;
    const uint4 *rl_rec;     // hubs' records (read when a block fills its table)
    const uint64_t *rl_rec8; // every vertex: id | offset << rl_sh_off | degree << rl_sh_deg
                             // (degree 0 for x < rl_fit, whose degree needs more bits)
    const uint32_t *rl_new;
    uint32_t rl_hubs;        // hubs of the plain relabel kernel (12 B each)
    uint32_t rl_sh_off, rl_sh_deg, rl_mask_id, rl_bits_deg;
    uint32_t rl_live, rl_fit;
    uint64_t rl_mask_off;
    bool compact() const { return rec8 != nullptr; }
};

// Device descriptors of AESC queries run as batches (batch.cu) or by the
// server (serve.cu).
struct GraphDesc {
    const int64_t *offsets;
    const uint32_t *nbrs;
    const uint2 *rec8;
    const uint64_t *upper_before;
    const uint4 *pk;
    const uint64_t *edge8;
    uint64_t mask_off;
    uint32_t n, pk_bits, pk_q, pk_mask, sh_off, sh_deg, mask_id, pad;
};

struct QueryDesc {
    GraphDesc g;
    uint64_t seed;
    const uint32_t *uv;
    const uint32_t *tau;
    const uint32_t *nwalks;
    uint32_t *counts;
    double *sc;
    uint64_t k;
    uint64_t ebase;  // first global edge index of this query
};

// Per queried edge: normalised endpoints, canonical id, degrees, plan.
struct BInfo {
    uint32_t u, v;
    uint64_t edge;
    uint32_t du, dv, tau, nwalks, valid, query;
};

// Up to kServeMany server requests in one prepare / scan / finalize launch
// (passed by value as the kernel parameter).
constexpr uint32_t kServeMany = 32;
struct ServeMany {
    const QueryDesc *qd[kServeMany];
    BInfo *info[kServeMany];
    uint32_t *tasks[kServeMany];
    uint64_t *begin[kServeMany];
    uint32_t *status[kServeMany];
    uint64_t edge_base[kServeMany + 1];
    uint32_t m;
};

// One in-flight request in a server iteration: its tasks [task_lo, task_lo +
// count) are work items [item_base, item_base + count) of the launch.
struct ServeItem {
    const QueryDesc *qd;
    const BInfo *info;
    const uint64_t *begin;
    uint64_t k;
    uint64_t task_lo;
    uint64_t item_base;
};

}  // namespace bq

struct bq_graph {
    int device = 0;
    uint32_t n = 0;
    uint64_t nnz = 0;
    int64_t *d_offsets = nullptr;
    uint32_t *d_nbrs = nullptr;
    bool owns_csr = true;
    uint2 *d_rec8 = nullptr;
    uint4 *d_rec16 = nullptr;
    uint64_t *d_upper_before = nullptr;
    uint64_t *d_edge8 = nullptr;
    uint4 *d_edge16 = nullptr;
    uint32_t sh_off = 0, sh_deg = 0, mask_id = 0;
    uint64_t mask_off = 0;
    uint4 *d_pk = nullptr;
    uint32_t pk_bits = 0, pk_q = 0, pk_mask = 0;
    int layout = 0;  // layout chosen at creation (bq_tuning.layout values)
    uint32_t *d_hub_tag = nullptr;
    uint32_t hub_slots = 0;
    uint32_t hub_cluster = 1;
    uint4 *d_rl_pk = nullptr;
    uint4 *d_rl_rec = nullptr;
    uint64_t *d_rl_rec8 = nullptr;
    uint32_t *d_rl_new = nullptr;
    uint32_t rl_hubs = 0;
    uint32_t rl_sh_off = 0, rl_sh_deg = 0, rl_mask_id = 0, rl_bits_deg = 0;
    uint32_t rl_live = 0;  // internal ids below this have neighbours
    uint32_t rl_fit = 0;   // internal ids from here on have their degree in rl_rec8
    uint64_t rl_mask_off = 0;
    uint32_t min_degree = 0, max_degree = 0;
    uint64_t m_upper = 0;  // entries v > u over all rows u (= m when symmetric)
    uint64_t device_bytes = 0;
    // lazily filled host copies / properties
    std::vector<int64_t> h_offsets;
    std::vector<uint32_t> h_nbrs;
    int bipartite = -1;
    int n_components = -1;
    bool has_spectrum = false;
    double lambda2 = 0.0, lambda_neg = 0.0;
    // omega known eigenpairs for the certified plan (bq_graph_set_eigvecs):
    // eigenvalues, eigenvectors scaled by 1/sqrt(d) (n x omega, row per
    // vertex), and the largest eigenvalue not given
    uint32_t omega = 0;
    std::vector<double> eig_lambdas, eig_vecs;
    double eig_rest = 0.0;

    bq::DeviceGraph view() const {
        bq::DeviceGraph v;
        v.n = n;
        v.nnz = nnz;
        v.offsets = d_offsets;
        v.nbrs = d_nbrs;
        v.rec8 = d_rec8;
        v.rec16 = d_rec16;
        v.upper_before = d_upper_before;
        v.edge8 = d_edge8;
        v.edge16 = d_edge16;
        v.sh_off = sh_off;
        v.sh_deg = sh_deg;
        v.mask_id = mask_id;
        v.mask_off = mask_off;
        v.pk = d_pk;
        v.pk_bits = pk_bits;
        v.pk_q = pk_q;
        v.pk_mask = pk_mask;
        v.hub_tag = d_hub_tag;
        v.hub_slots = hub_slots;
        v.hub_cluster = hub_cluster;
        v.rl_pk = d_rl_pk;
        v.rl_rec = d_rl_rec;
        v.rl_rec8 = d_rl_rec8;
        v.rl_sh_off = rl_sh_off;
        v.rl_sh_deg = rl_sh_deg;
        v.rl_mask_id = rl_mask_id;
        v.rl_mask_off = rl_mask_off;
        v.rl_new = d_rl_new;
        v.rl_hubs = rl_hubs;
        v.rl_bits_deg = rl_bits_deg;
        v.rl_live = rl_live;
        v.rl_fit = rl_fit;
        return v;
    }
};

namespace bq {

// ---- NVTX: a named range over each library call and server iteration
// (shown by Nsight tools; a no-op when none is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Makes `dev` the current device for a scope, then restores the previous one.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

// ---- error plumbing (api.cu)
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t err, const char *what);
void clear_error();  // empties this thread's bq_last_error() message
// scheduled plan of one edge (api.cu; shared by bq_aesc_plan and the server)
void plan_scheduled_edge(double s_e, double eps, const bq_schedule &sched, uint32_t &tau, double &nw);
#define BQ_CUDA(call)                                            \
    do {                                                         \
        cudaError_t _e = (call);                                 \
        if (_e != cudaSuccess) return ::bq::cuda_fail(_e, #call); \
    } while (0)

// Per-device status word (allocated on first graph creation on a device).
int status_word(int device, uint32_t **out);

// Device-pool allocation helpers on a stream.
int scratch_alloc(void **p, size_t bytes, cudaStream_t s);
void scratch_free(void *p, cudaStream_t s);

// Performance knobs (never change a result): walks per lane of the bouquet
// walk-batch kernel (1, 2, 4, 8), warp-aggregated visit atomics, walks per
// lane of the AESC counting kernel (2, 4, 8).
int tuning_walks_per_lane();
bool tuning_aggregate_visits();
int tuning_aesc_walks_per_lane();
int tuning_layout();    // graph layout built at creation (bq_tuning.layout)
int tuning_hub_slots();  // hub table size built at creation (bq_tuning.hub_slots)
int tuning_hub_cluster();  // CTAs a created graph's hub table is spread over
bool tuning_hub_relabel();  // created packed-id graphs get the degree-relabelled copy
bool tuning_l2_hints(); // L2 eviction policies on the walk kernel's loads
bool tuning_aesc_hub();  // AESC counting reads hub records from shared memory
bool tuning_relabel_hub8();      // relabelled copy: 8-byte hubs (else the 12-byte relabel kernel)
uint32_t tuning_hub8_hubs();       // their number (0: what the 12-byte kernel's shared memory holds)
uint32_t tuning_hub8_count_bits(); // cap on their count-field width (0: every bit above the id)
int tuning_shared_lanes();         // walks per lane of the vertex-centric kernels (2, 4, 8)
int tuning_push_walks_per_lane();  // walks per lane of the push-phase counting kernel
bool tuning_group_walks();         // walk batches group their walks by start vertex (bouquets)

// Profiling (api.cu): event brackets around kernel groups while enabled, and
// a count of every kernel launch.
enum ProfKind { kProfWalk = 0, kProfGroup = 1, kProfAesc = 2, kProfAescAux = 3 };
struct ProfScope {
    int kind;
    cudaStream_t stream;
    cudaEvent_t start = nullptr, stop = nullptr;
    ProfScope(int kind, cudaStream_t s);
    ~ProfScope();
};
void count_launches(unsigned n);
void count_walk_kernel(int kind);  // BQ_WALK_KERNEL_* of a walk-batch launch

// ---- graph.cu
// Validate a device CSR and build records / edge numbering.  Synchronous on s.
int graph_build(bq_graph *g, uint32_t flags, cudaStream_t s);
// Exclusive scan of uint32 counts into uint64 prefix (out has n + 1 entries).
int scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, cudaStream_t s);
// Exclusive scan of uint32 into uint32 (out has n + 1 entries; caller
// guarantees the total fits).
int scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, cudaStream_t s);
// Copy the CSR to the host copies of g (once).
int graph_fetch_host(bq_graph *g);

// ---- walks.cu
int launch_walk_batch(const DeviceGraph &g, uint64_t seed, const uint32_t *starts,
                      uint64_t n_walks, uint32_t n_steps, uint32_t mode,
                      const Sampler &smp, bool visit_start, uint32_t *visits,
                      uint32_t *paths, uint32_t *status, cudaStream_t s);

// Bouquet walk batch in a caller-provided scratch region (no allocation).
size_t walk_batch_scratch_bytes(uint32_t n, uint64_t n_walks);
int launch_walk_batch_in(const DeviceGraph &g, uint64_t seed, const uint32_t *starts, uint64_t n_walks,
                         uint32_t n_steps, const Sampler &smp, bool visit_start, uint32_t *visits, uint32_t *paths,
                         uint32_t *status, void *scratch, size_t scratch_bytes, cudaStream_t s);
// graph.cu: the scan with its tile sums in a caller workspace.
size_t scan_u32_ws_bytes(uint64_t n);
int scan_u32_ws(const uint32_t *in, uint32_t *out, uint64_t n, void *ws, size_t ws_bytes, cudaStream_t s);
size_t scan_u32_to_u64_ws_bytes(uint64_t n);
int scan_u32_to_u64_ws(const uint32_t *in, uint64_t *out, uint64_t n, void *ws, size_t ws_bytes, cudaStream_t s);
// api.cu: the device's status word if it was already allocated (never allocates).
int existing_status_word(int device, uint32_t **out);
int validate_sampler(const bq_sampler *in, Sampler &out, bool allow_saba = false);

// ---- batch.cu, used by the server: one query's edges (prepare + task scan),
// an iteration over windows of several queries' tasks, and the finalize.
GraphDesc graph_desc(const bq_graph *g);
int serve_iterate(const ServeItem *d_items, uint32_t n_items, uint64_t total_items, int lanes, const Sampler &smp,
                  unsigned long long *counter, cudaStream_t s);
// prepare + task scan, or finalize, of up to kServeMany requests in one launch each
int serve_prepare_many(const ServeMany &L, uint32_t bouquet, cudaStream_t s);
int serve_finalize_many(const ServeMany &L, cudaStream_t s);

// ---- shared.cu: batches of vertex-centric estimates (bq_batch_create_shared)
struct SharedBatch;
int shared_batch_create(const bq_aesc_query *queries, uint32_t n_queries, const Sampler &smp, SharedBatch **out,
                        uint64_t *edges);
int shared_batch_run(SharedBatch *b, cudaStream_t s);
void shared_batch_free(SharedBatch *b);

// ---- aesc.cu
// naive: one walk per thread on the plain CSR (BQ_AESC_NAIVE), else bouquets
int launch_aesc(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv,
                uint64_t k, const uint32_t *tau, const uint32_t *nwalks,
                const Sampler &smp, bool naive, uint32_t *counts, double *sc, uint32_t *status,
                cudaStream_t s);
// Pilot of the scheduled plan: per query and side the sums of a, b, a^2,
// b^2, a b over the first nwalks[q] walks (a, b = one walk's weighted hits of
// u and of v) into moments = device uint64[10k]; edges_uv explicit.  With
// pilot != NULL (nwalks[q] = pilot->n0 for all q) the walk count of the pilot
// plan is then written to nwalks_out (device uint32[k]).
struct PilotParams {
    uint32_t n0;
    uint32_t n_min;
    double eps, z;
};
int launch_aesc_moments(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k,
                        const uint32_t *tau, const uint32_t *nwalks, const Sampler &smp, uint64_t *moments,
                        const PilotParams *pilot, uint32_t *nwalks_out, uint32_t *status, cudaStream_t s);
// Canonical edge list (edges ordered by lower endpoint, then higher) into
// uv = device uint32[2m].
int launch_canonical_edges(const DeviceGraph &g, uint32_t *uv, cudaStream_t s);
// support_cap: 1..kPushSupportCapMax, the largest support per side and level
// admitted at push depths >= 2
constexpr uint32_t kPushSupportCapMax = 512;
int launch_aesc_push(const DeviceGraph &g, uint64_t seed, const uint32_t *edges_uv, uint64_t k,
                     const uint32_t *tau, const uint32_t *nwalks, uint32_t push_max, uint32_t support_cap,
                     uint32_t *depth_out, uint64_t *acc, double *sc, uint32_t *status, cudaStream_t s);

}  // namespace bq
