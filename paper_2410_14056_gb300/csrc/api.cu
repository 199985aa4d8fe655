// C-ABI entry points of libbouquet (declared in include/bouquet.h): argument
// checking, host-side staging for BQ_HOST_IO calls, the host planner, the
// per-device status word, and error reporting.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace bq {

namespace {
thread_local char g_last_error[1024] = "";
std::mutex g_dev_mutex;
std::vector<uint32_t *> g_status;       // per device ordinal
std::vector<char> g_pool_configured;    // per device ordinal

std::atomic<int> g_walks_per_lane{4};
std::atomic<int> g_aggregate{0};
std::atomic<int> g_aesc_walks_per_lane{4};
std::atomic<int> g_edge_records{1};
std::atomic<int> g_hub_slots{8192};
std::atomic<int> g_hub_cluster{1};
std::atomic<int> g_hub_relabel{0};
std::atomic<int> g_l2_hints{0};
std::atomic<int> g_aesc_hub{0};
std::atomic<int> g_relabel_hub8{1};
std::atomic<int> g_hub8_hubs{0};
std::atomic<int> g_hub8_count_bits{0};
std::atomic<int> g_shared_lanes{2};
std::atomic<int> g_group_walks{1};
std::atomic<int> g_push_lanes{2};
}  // namespace

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_last_error[0] = 0; }

int cuda_fail(cudaError_t err, const char *what) {
    return fail(BQ_ECUDA, "%s: %s (%s)", what, cudaGetErrorString(err), cudaGetErrorName(err));
}

int status_word(int device, uint32_t **out) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if ((int)g_status.size() <= device) {
        g_status.resize(device + 1, nullptr);
        g_pool_configured.resize(device + 1, 0);
    }
    if (!g_status[device]) {
        uint32_t *p = nullptr;
        BQ_CUDA(cudaMalloc(&p, sizeof(uint32_t)));
        BQ_CUDA(cudaMemset(p, 0, sizeof(uint32_t)));
        g_status[device] = p;
    }
    if (!g_pool_configured[device]) {
        // Keep freed scratch in the device's default pool between calls
        // instead of returning it to the driver at every synchronisation.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        g_pool_configured[device] = 1;
    }
    *out = g_status[device];
    return BQ_OK;
}

int existing_status_word(int device, uint32_t **out) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if ((int)g_status.size() <= device || !g_status[device])
        return fail(BQ_EINVAL, "no status word on device %d: create a graph on it first", device);
    *out = g_status[device];
    return BQ_OK;
}

int scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(BQ_ENOMEM, "cannot allocate %zu bytes of device scratch", bytes);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    return BQ_OK;
}

void scratch_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------- profiling

namespace {
struct PendingTiming {
    int kind;
    cudaEvent_t start, stop;
};
std::mutex g_prof_mutex;
std::atomic<int> g_prof_enabled{0};
std::vector<PendingTiming> g_prof_pending;
std::vector<cudaEvent_t> g_prof_free_events;
double g_prof_ms[4] = {0, 0, 0, 0};
uint64_t g_prof_count[4] = {0, 0, 0, 0};
std::atomic<uint64_t> g_launches{0};
std::atomic<uint64_t> g_walk_kernels[8];

cudaEvent_t take_event() {
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (!g_prof_free_events.empty()) {
        cudaEvent_t e = g_prof_free_events.back();
        g_prof_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

ProfScope::ProfScope(int k, cudaStream_t s) : kind(k), stream(s) {
    if (!g_prof_enabled.load()) return;
    start = take_event();
    stop = take_event();
    if (start && stop) cudaEventRecord(start, s);
}

ProfScope::~ProfScope() {
    if (!start || !stop) return;
    cudaEventRecord(stop, stream);
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    g_prof_pending.push_back(PendingTiming{kind, start, stop});
}

void count_launches(unsigned n) { g_launches.fetch_add(n); }
void count_walk_kernel(int kind) {
    if (kind >= 0 && kind < 8) g_walk_kernels[kind].fetch_add(1);
}

int validate_sampler(const bq_sampler *in, Sampler &out);

int tuning_walks_per_lane() { return g_walks_per_lane.load(); }
bool tuning_aggregate_visits() { return g_aggregate.load() != 0; }
int tuning_aesc_walks_per_lane() { return g_aesc_walks_per_lane.load(); }
int tuning_layout() { return g_edge_records.load(); }
int tuning_hub_slots() { return g_hub_slots.load(); }
int tuning_hub_cluster() { return g_hub_cluster.load(); }
bool tuning_hub_relabel() { return g_hub_relabel.load() != 0; }
bool tuning_l2_hints() { return g_l2_hints.load() != 0; }
bool tuning_aesc_hub() { return g_aesc_hub.load() != 0; }
bool tuning_relabel_hub8() { return g_relabel_hub8.load() != 0; }
uint32_t tuning_hub8_hubs() { return (uint32_t)g_hub8_hubs.load(); }
uint32_t tuning_hub8_count_bits() { return (uint32_t)g_hub8_count_bits.load(); }
int tuning_shared_lanes() { return g_shared_lanes.load(); }
bool tuning_group_walks() { return g_group_walks.load() != 0; }
int tuning_push_walks_per_lane() { return g_push_lanes.load(); }

namespace {

// The literal SABA word (walk batches only) runs on the coupled path with
// t = kSabaT and one group for the whole batch.
int check_sampler(const bq_sampler *in, Sampler &out, bool allow_saba = false) {
    out.kind = 0;
    out.t = 0;
    out.width = 1;
    if (!in) return BQ_OK;
    if (in->kind == BQ_SAMPLER_IND) return BQ_OK;
    if (in->kind == BQ_SAMPLER_SABA) {
        if (!allow_saba) return fail(BQ_EINVAL, "the literal SABA sampler is for walk batches only");
        out.kind = 1;
        out.t = kSabaT;
        out.width = 1;
        return BQ_OK;
    }
    if (in->kind != BQ_SAMPLER_COUPLED) return fail(BQ_EINVAL, "unknown sampler kind %u", in->kind);
    if (in->width < 1) return fail(BQ_EINVAL, "coupled sampler needs width >= 1");
    if (in->t > 32) return fail(BQ_EINVAL, "coupled sampler needs 0 <= t <= 32 (got %u)", in->t);
    out.kind = 1;
    out.t = in->t;
    out.width = in->width;
    return BQ_OK;
}

// Components and 2-colourability by BFS over the host copy of the CSR.
void host_structure(bq_graph *g) {
    if (g->n_components >= 0) return;
    const uint32_t n = g->n;
    std::vector<int8_t> color(n, -1);
    std::vector<uint32_t> queue;
    queue.reserve(1024);
    int comps = 0;
    bool bip = true;
    for (uint32_t s = 0; s < n; ++s) {
        if (color[s] >= 0) continue;
        ++comps;
        color[s] = 0;
        queue.clear();
        queue.push_back(s);
        for (size_t h = 0; h < queue.size(); ++h) {
            const uint32_t x = queue[h];
            for (int64_t j = g->h_offsets[x]; j < g->h_offsets[x + 1]; ++j) {
                const uint32_t y = g->h_nbrs[j];
                if (color[y] < 0) {
                    color[y] = (int8_t)(1 - color[x]);
                    queue.push_back(y);
                } else if (color[y] == color[x]) {
                    bip = false;
                }
            }
        }
    }
    g->n_components = comps;
    g->bipartite = bip ? 1 : 0;
}

}  // namespace

int validate_sampler(const bq_sampler *in, Sampler &out, bool allow_saba) {
    return check_sampler(in, out, allow_saba);
}

}  // namespace bq

using namespace bq;

extern "C" {

const char *bq_version(void) { return "bouquet-gb300 0.2"; }

const char *bq_last_error(void) { return g_last_error; }

const char *bq_strerror(int code) {
    switch (code) {
    case BQ_OK: return "ok";
    case BQ_EINVAL: return "invalid argument";
    case BQ_ENOMEM: return "out of memory";
    case BQ_EGRAPH: return "graph rejected by validation";
    case BQ_ENOEDGE: return "vertex pair is not an edge";
    case BQ_EOVERFLOW: return "counter or plan overflow";
    case BQ_ETIMEOUT: return "bounded wait timed out";
    case BQ_EBUSY: return "admission refused";
    case BQ_ECUDA: return "CUDA runtime error";
    default: return "unknown status code";
    }
}

int bq_graph_create(uint32_t n, const int64_t *offsets, const uint32_t *nbrs, uint32_t flags, void *cuda_stream,
                    bq_graph **out) {
    bq::NvtxRange nvtx_range("bq_graph_create");
    g_last_error[0] = 0;
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!offsets) return fail(BQ_EINVAL, "offsets is NULL");
    if (flags & ~(BQ_DEVICE_PTRS | BQ_BORROW | BQ_SKIP_VALIDATE | BQ_REQUIRE_CONNECTED))
        return fail(BQ_EINVAL, "unknown graph flags 0x%x", flags);
    if ((flags & BQ_BORROW) && !(flags & BQ_DEVICE_PTRS))
        return fail(BQ_EINVAL, "BQ_BORROW requires BQ_DEVICE_PTRS");
    if (n == 0xffffffffu) return fail(BQ_EINVAL, "n must be < 2^32 - 1");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int dev = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    uint32_t *status = nullptr;
    int rc = status_word(dev, &status);
    if (rc) return rc;

    // nnz = offsets[n]
    int64_t nnz = 0;
    if (flags & BQ_DEVICE_PTRS) {
        BQ_CUDA(cudaMemcpyAsync(&nnz, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BQ_CUDA(cudaStreamSynchronize(s));
    } else {
        nnz = offsets[n];
    }
    if (nnz < 0) return fail(BQ_EGRAPH, "offsets[n] = %lld is negative", (long long)nnz);
    if (nnz > 0 && !nbrs) return fail(BQ_EINVAL, "nbrs is NULL");

    bq_graph *g = new (std::nothrow) bq_graph();
    if (!g) return fail(BQ_ENOMEM, "host allocation failed");
    g->device = dev;
    g->n = n;
    g->nnz = (uint64_t)nnz;
    cudaError_t e = cudaSuccess;
    if (flags & BQ_BORROW) {
        g->owns_csr = false;
        g->d_offsets = const_cast<int64_t *>(offsets);
        g->d_nbrs = const_cast<uint32_t *>(nbrs);
    } else {
        const cudaMemcpyKind kind = (flags & BQ_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = cudaMalloc(&g->d_offsets, sizeof(int64_t) * ((size_t)n + 1));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_nbrs, sizeof(uint32_t) * std::max<uint64_t>(g->nnz, 1));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(g->d_offsets, offsets, sizeof(int64_t) * ((size_t)n + 1), kind, s);
        if (e == cudaSuccess && g->nnz)
            e = cudaMemcpyAsync(g->d_nbrs, nbrs, sizeof(uint32_t) * g->nnz, kind, s);
        if (e != cudaSuccess) {
            rc = (e == cudaErrorMemoryAllocation) ? fail(BQ_ENOMEM, "cannot allocate the device CSR")
                                                  : cuda_fail(e, "graph upload");
            bq_graph_destroy(g);
            return rc;
        }
        g->device_bytes += sizeof(int64_t) * ((size_t)n + 1) + sizeof(uint32_t) * g->nnz;
    }
    rc = graph_build(g, flags, s);
    if (rc == BQ_OK && (flags & BQ_REQUIRE_CONNECTED)) {
        rc = graph_fetch_host(g);
        if (rc == BQ_OK) {
            host_structure(g);
            if (g->n_components > 1)
                rc = fail(BQ_EGRAPH, "graph has %d connected components (BQ_REQUIRE_CONNECTED)", g->n_components);
        }
    }
    if (rc != BQ_OK) {
        bq_graph_destroy(g);
        return rc;
    }
    *out = g;
    return BQ_OK;
}

int bq_graph_destroy(bq_graph *g) {
    if (!g) return BQ_OK;
    DeviceGuard guard(g->device);
    if (g->owns_csr) {
        cudaFree(g->d_offsets);
        cudaFree(g->d_nbrs);
    }
    cudaFree(g->d_rec8);
    cudaFree(g->d_rec16);
    cudaFree(g->d_upper_before);
    cudaFree(g->d_edge8);
    cudaFree(g->d_edge16);
    cudaFree(g->d_pk);
    cudaFree(g->d_rl_pk);
    cudaFree(g->d_rl_rec);
    cudaFree(g->d_rl_rec8);
    cudaFree(g->d_rl_new);
    cudaFree(g->d_hub_tag);
    delete g;
    return BQ_OK;
}

int bq_graph_info(bq_graph *g, bq_graph_info_t *info) {
    g_last_error[0] = 0;
    if (!g || !info) return fail(BQ_EINVAL, "NULL argument");
    int rc = graph_fetch_host(g);
    if (rc) return rc;
    host_structure(g);
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->nnz = g->nnz;
    info->m = g->nnz / 2;
    info->min_degree = g->n ? g->min_degree : 0;
    info->max_degree = g->max_degree;
    info->bipartite = g->bipartite;
    info->n_components = g->n_components;
    info->device_bytes = g->device_bytes;
    info->has_spectrum = g->has_spectrum ? 1 : 0;
    info->device = g->device;
    info->lambda2 = g->lambda2;
    info->lambda_neg = g->lambda_neg;
    info->layout = g->layout;
    info->hub_slots = g->d_hub_tag ? g->hub_slots * g->hub_cluster : 0;
    info->packed_bits = g->d_pk ? g->pk_bits : 0;
    if (g->d_rl_pk) {
        info->relabel_hubs = g->rl_hubs;
        info->relabel_bits_id = g->rl_sh_off;
        info->relabel_bits_off = g->rl_sh_deg - g->rl_sh_off;
        info->relabel_bits_deg = g->rl_bits_deg;
    }
    return BQ_OK;
}

int bq_graph_set_spectrum(bq_graph *g, double lambda2, double lambda_neg) {
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (!(lambda2 < 1.0) || !(lambda2 >= -1.0)) return fail(BQ_EINVAL, "lambda2 = %g must lie in [-1, 1)", lambda2);
    if (!(lambda_neg <= 0.0) || !(lambda_neg >= -1.0))
        return fail(BQ_EINVAL, "lambda_neg = %g must lie in [-1, 0]", lambda_neg);
    g->lambda2 = lambda2;
    g->lambda_neg = lambda_neg;
    g->has_spectrum = true;
    return BQ_OK;
}

int bq_graph_set_eigvecs(bq_graph *g, uint32_t omega, const double *lambdas, const double *vecs,
                         double lambda_rest) {
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (omega == 0) {
        g->omega = 0;
        g->eig_lambdas.clear();
        g->eig_vecs.clear();
        g->eig_rest = 0.0;
        return BQ_OK;
    }
    if (!lambdas || !vecs) return fail(BQ_EINVAL, "lambdas or vecs is NULL");
    if (omega >= g->n) return fail(BQ_EINVAL, "omega = %u must be below n = %u", omega, g->n);
    for (uint32_t j = 0; j < omega; ++j)
        if (!(lambdas[j] < 1.0) || !(lambdas[j] >= -1.0))
            return fail(BQ_EINVAL, "eigenvalue %u = %g must lie in [-1, 1)", j, lambdas[j]);
    if (!(lambda_rest < 1.0) || !(lambda_rest >= -1.0))
        return fail(BQ_EINVAL, "lambda_rest = %g must lie in [-1, 1)", lambda_rest);
    const size_t count = (size_t)g->n * omega;
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(vecs[i])) return fail(BQ_EINVAL, "vecs[%zu] is not finite", i);
    g->eig_lambdas.assign(lambdas, lambdas + omega);
    g->eig_vecs.assign(vecs, vecs + count);
    g->eig_rest = lambda_rest;
    g->omega = omega;
    return BQ_OK;
}

int bq_walk_batch(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev, uint64_t n_walks, uint32_t n_steps,
                  uint32_t mode, const bq_sampler *sampler, uint32_t flags, uint32_t *visits_dev, uint32_t *paths_dev,
                  void *stream) {
    bq::NvtxRange nvtx_range("bq_walk_batch");
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (mode != BQ_MODE_NAIVE && mode != BQ_MODE_BOUQUET) return fail(BQ_EINVAL, "unknown mode %u", mode);
    if (flags & ~(BQ_VISIT_START | BQ_HOST_IO)) return fail(BQ_EINVAL, "unknown walk flags 0x%x", flags);
    if (n_walks && (!starts_dev || !visits_dev)) return fail(BQ_EINVAL, "starts or visits is NULL");
    if (mode == BQ_MODE_BOUQUET && n_walks >= (1ull << 32))
        return fail(BQ_EINVAL, "bouquet mode takes fewer than 2^32 walks per call (got %llu)",
                    (unsigned long long)n_walks);
    if (paths_dev && n_walks > UINT64_MAX / ((uint64_t)n_steps + 1) / sizeof(uint32_t))
        return fail(BQ_EINVAL, "paths array size overflows");
    Sampler smp;
    int rc = check_sampler(sampler, smp, true);
    if (rc) return rc;
    if (n_walks == 0) return BQ_OK;
    DeviceGuard guard(g->device);
    uint32_t *status = nullptr;
    rc = status_word(g->device, &status);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool visit_start = (flags & BQ_VISIT_START) != 0;
    if (!(flags & BQ_HOST_IO))
        return launch_walk_batch(g->view(), seed, starts_dev, n_walks, n_steps, mode, smp, visit_start, visits_dev,
                                 paths_dev, status, s);

    // Host buffers: stage through stream-ordered device scratch.
    const size_t sb = sizeof(uint32_t) * n_walks, vb = sizeof(uint32_t) * g->n;
    const size_t pb = paths_dev ? sizeof(uint32_t) * n_walks * ((size_t)n_steps + 1) : 0;
    char *buf = nullptr;
    rc = scratch_alloc((void **)&buf, sb + vb + pb, s);
    if (rc) return rc;
    uint32_t *d_starts = (uint32_t *)buf, *d_visits = (uint32_t *)(buf + sb);
    uint32_t *d_paths = paths_dev ? (uint32_t *)(buf + sb + vb) : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_starts, starts_dev, sb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_visits, visits_dev, vb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "host-io upload");
    if (rc == BQ_OK)
        rc = launch_walk_batch(g->view(), seed, d_starts, n_walks, n_steps, mode, smp, visit_start, d_visits, d_paths,
                               status, s);
    if (rc == BQ_OK) {
        e = cudaMemcpyAsync(visits_dev, d_visits, vb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && d_paths) e = cudaMemcpyAsync(paths_dev, d_paths, pb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "host-io download");
    }
    scratch_free(buf, s);
    if (rc == BQ_OK) rc = bq_sync(stream);
    else cudaStreamSynchronize(s);
    return rc;
}

// ------------------------------------------------------------- planner

namespace {

double trunc_factor(double lambda2, double lambda_neg, uint32_t tau) {
    // worst eigen-component error factor lambda^tau (1+lambda)/(2(1-lambda))
    double pos = 0.0, neg = 0.0;
    if (lambda2 > 0.0) pos = pow(lambda2, (double)tau) * (1.0 + lambda2) / (2.0 * (1.0 - lambda2));
    const double a = -lambda_neg;
    if (a > 0.0) {
        // maximiser of x^tau (1-x)/(1+x): root of tau x^2 + 2x - tau = 0
        const double peak = (sqrt(1.0 + (double)tau * (double)tau) - 1.0) / (double)tau;
        const double x = std::min(a, peak);
        neg = pow(x, (double)tau) * (1.0 - x) / (2.0 * (1.0 + x));
    }
    return std::max(pos, neg);
}

// Truncation bound with the graph's omega known eigenpairs: the known modes'
// error sum_k c_k^2 lambda_k^tau (1 + lambda_k) / (2 (1 - lambda_k)) exactly
// (c_k = psi_k(u)/sqrt(d_u) - psi_k(v)/sqrt(d_v)), the remaining mass
// s_e - sum_k c_k^2 times the worst factor of the eigenvalues not given.
double trunc_bound_omega(const bq_graph *g, uint32_t u, uint32_t v, double s_e, uint32_t tau) {
    const uint32_t w = g->omega;
    const double *cu = g->eig_vecs.data() + (size_t)u * w;
    const double *cv = g->eig_vecs.data() + (size_t)v * w;
    double known = 0.0, mass = 0.0;
    for (uint32_t j = 0; j < w; ++j) {
        const double c = cu[j] - cv[j], l = g->eig_lambdas[j];
        known += c * c * pow(l, (double)tau) * (1.0 + l) / (2.0 * (1.0 - l));
        mass += c * c;
    }
    double rest = s_e - mass;
    if (rest < 0.0) rest = 0.0;
    return fabs(known) + rest * trunc_factor(g->eig_rest, g->lambda_neg, tau);
}

// Position of v in the sorted row of u, or -1.
int64_t find_in_row(const bq_graph *g, uint32_t u, uint32_t v) {
    const uint32_t *b = g->h_nbrs.data() + g->h_offsets[u];
    const uint32_t *e = g->h_nbrs.data() + g->h_offsets[u + 1];
    const uint32_t *p = std::lower_bound(b, e, v);
    return (p != e && *p == v) ? (int64_t)(p - b) : -1;
}

}  // namespace

}  // extern "C"

namespace bq {

// Scheduled plan of one edge (s_e = 1/d_u + 1/d_v): tau = clamp(ceil(c ln(s_e /
// eps)) + a, 1, tau_max) with the log term only when s_e > eps, N =
// max(N_min, ceil(k s_e^2 / eps^2)).
void plan_scheduled_edge(double s_e, double eps, const bq_schedule &sched, uint32_t &tau, double &nw) {
    const double ratio = s_e / eps;
    double tt = ratio > 1.0 ? ceil(sched.tau_scale * log(ratio)) : 0.0;
    tt += (double)sched.tau_add;
    if (tt < 1.0) tt = 1.0;
    if (tt > (double)sched.tau_max) tt = (double)sched.tau_max;
    tau = (uint32_t)tt;
    nw = ceil(sched.n_scale * s_e * s_e / (eps * eps));
    if (nw < (double)sched.n_min) nw = (double)sched.n_min;
}

// Run f(begin, end) over [0, count) on up to 16 host threads (one thread
// for small counts).
template <typename F>
void parallel_ranges(uint64_t count, F &&f) {
    unsigned threads = std::thread::hardware_concurrency();
    if (threads < 1) threads = 1;
    if (threads > 16) threads = 16;
    if (count < (1u << 16) || threads == 1) {
        f((uint64_t)0, count);
        return;
    }
    std::vector<std::thread> pool;
    const uint64_t per = (count + threads - 1) / threads;
    for (unsigned i = 0; i < threads; ++i) {
        const uint64_t b = (uint64_t)i * per, e = std::min(count, b + per);
        if (b >= e) break;
        pool.emplace_back([&f, b, e] { f(b, e); });
    }
    for (auto &t : pool) t.join();
}

// The canonical pairs {u, v}, u < v, of every edge in row order (the
// library's edge numbering), built in two parallel passes over the rows;
// false when the rows are not symmetric.
bool canonical_pairs_host(const bq_graph *g, std::vector<uint32_t> &canon) {
    const uint64_t n = g->n;
    std::vector<uint64_t> start(n + 1, 0);
    parallel_ranges(n, [&](uint64_t b, uint64_t e) {
        for (uint64_t u = b; u < e; ++u) {
            uint64_t c = 0;
            for (int64_t j = g->h_offsets[u]; j < g->h_offsets[u + 1]; ++j) c += g->h_nbrs[j] > u ? 1 : 0;
            start[u + 1] = c;
        }
    });
    for (uint64_t u = 0; u < n; ++u) start[u + 1] += start[u];
    if (start[n] != g->nnz / 2) return false;
    canon.resize(2 * start[n]);
    parallel_ranges(n, [&](uint64_t b, uint64_t e) {
        for (uint64_t u = b; u < e; ++u) {
            uint64_t p = start[u];
            for (int64_t j = g->h_offsets[u]; j < g->h_offsets[u + 1]; ++j)
                if (g->h_nbrs[j] > u) {
                    canon[2 * p] = (uint32_t)u;
                    canon[2 * p + 1] = g->h_nbrs[j];
                    ++p;
                }
        }
    });
    return true;
}

}  // namespace bq

extern "C" {

int bq_aesc_plan(bq_graph *g, const uint32_t *edges_uv, uint64_t k, double eps, double delta, uint32_t plan_mode,
                 const bq_schedule *sched, uint32_t *tau, uint32_t *nwalks) {
    bq::NvtxRange nvtx_range("bq_aesc_plan");
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (!(eps > 0.0) || !(eps < 1e6)) return fail(BQ_EINVAL, "eps = %g must be positive", eps);
    if (k && (!tau || !nwalks)) return fail(BQ_EINVAL, "tau or nwalks is NULL");
    const uint64_t m = g->nnz / 2;
    if (!edges_uv && k != m)
        return fail(BQ_EINVAL, "all-edges plan needs k = m = %llu (got %llu)", (unsigned long long)m,
                    (unsigned long long)k);
    if (plan_mode == BQ_PLAN_CERTIFIED) {
        if (!(delta > 0.0) || !(delta < 1.0)) return fail(BQ_EINVAL, "delta = %g must lie in (0, 1)", delta);
        if (!g->has_spectrum) return fail(BQ_EINVAL, "certified plan needs bq_graph_set_spectrum first");
    } else if (plan_mode == BQ_PLAN_SCHEDULED) {
        if (!sched) return fail(BQ_EINVAL, "scheduled plan needs a schedule");
        if (sched->tau_max < 1 || !(sched->tau_scale >= 0.0) || !(sched->n_scale >= 0.0))
            return fail(BQ_EINVAL, "bad schedule");
    } else {
        return fail(BQ_EINVAL, "unknown plan mode %u", plan_mode);
    }
    if (k == 0) return BQ_OK;
    int rc = graph_fetch_host(g);
    if (rc) return rc;
    const double log_term = plan_mode == BQ_PLAN_CERTIFIED ? log(2.0 * (double)m / delta) : 0.0;
    // all-edges plan: canonical order = rows in order, neighbours above the row
    std::vector<uint32_t> canon;
    if (!edges_uv && !canonical_pairs_host(g, canon)) return fail(BQ_EGRAPH, "graph is not symmetric");
    const uint32_t *pairs = edges_uv ? edges_uv : canon.data();
    // per-edge plans on host threads; each range stops at its first failing
    // query, and the lowest failing query is reported (as a serial loop would)
    struct PlanError {
        uint64_t q = UINT64_MAX;
        int kind = 0;  // 0 not an edge, 1 tau cap, 2 2 N tau >= 2^32
        uint32_t a = 0, b = 0;
        double value = 0.0;
    };
    const uint32_t tau_cap = 1u << 20;
    std::mutex err_mutex;
    PlanError first;
    parallel_ranges(k, [&](uint64_t begin, uint64_t end) {
        PlanError err;
        for (uint64_t q = begin; q < end && err.q == UINT64_MAX; ++q) {
            const uint32_t a = pairs[2 * q], b = pairs[2 * q + 1];
            if (edges_uv && (a >= g->n || b >= g->n || a == b || find_in_row(g, a, b) < 0)) {
                err.q = q;
                err.kind = 0;
                err.a = a;
                err.b = b;
                break;
            }
            const double du = (double)(g->h_offsets[a + 1] - g->h_offsets[a]);
            const double dv = (double)(g->h_offsets[b + 1] - g->h_offsets[b]);
            const double s_e = 1.0 / du + 1.0 / dv;
            uint32_t t = 1;
            double nw = 0.0;
            if (plan_mode == BQ_PLAN_CERTIFIED) {
                while ((g->omega ? trunc_bound_omega(g, a, b, s_e, t)
                                 : s_e * trunc_factor(g->lambda2, g->lambda_neg, t)) > eps / 2.0) {
                    if (t >= tau_cap) {
                        err.q = q;
                        err.kind = 1;
                        break;
                    }
                    ++t;
                }
                if (err.q != UINT64_MAX) break;
                const double half = (double)t - 0.5;
                nw = ceil(8.0 * half * half * s_e * s_e * log_term / (eps * eps));
            } else {
                plan_scheduled_edge(s_e, eps, *sched, t, nw);
            }
            if (nw < 1.0) nw = 1.0;
            if (nw * 2.0 * (double)t >= 4294967296.0) {
                err.q = q;
                err.kind = 2;
                err.value = nw * 2.0 * (double)t;
                break;
            }
            tau[q] = t;
            nwalks[q] = (uint32_t)nw;
        }
        if (err.q != UINT64_MAX) {
            std::lock_guard<std::mutex> lock(err_mutex);
            if (err.q < first.q) first = err;
        }
    });
    if (first.q != UINT64_MAX) {
        const unsigned long long q = (unsigned long long)first.q;
        if (first.kind == 0) return fail(BQ_ENOEDGE, "query %llu: (%u, %u) is not an edge", q, first.a, first.b);
        if (first.kind == 1) return fail(BQ_EOVERFLOW, "query %llu: truncation length exceeds %u", q, tau_cap);
        return fail(BQ_EOVERFLOW, "query %llu: 2 * N * tau = %.3g reaches 2^32", q, first.value);
    }
    return BQ_OK;
}

int bq_aesc_plan_pilot(bq_graph *g, uint64_t seed, const uint32_t *edges_uv, uint64_t k, double eps,
                       const bq_schedule *sched, uint32_t n_pilot, double z, const bq_sampler *sampler,
                       uint32_t *tau, uint32_t *nwalks, uint64_t *moments, void *stream) {
    bq::NvtxRange nvtx_range("bq_aesc_plan_pilot");
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (!sched) return fail(BQ_EINVAL, "pilot plan needs a schedule");
    if (n_pilot < 2) return fail(BQ_EINVAL, "n_pilot = %u (at least 2)", n_pilot);
    if (!(z > 0.0) || !(z < 1e6)) return fail(BQ_EINVAL, "z = %g must be positive", z);
    Sampler smp;
    int rc = check_sampler(sampler, smp);
    if (rc) return rc;
    // tau from the schedule (its N part unused: n_scale 0, n_min 1)
    bq_schedule tau_only = *sched;
    tau_only.n_scale = 0.0;
    tau_only.n_min = 1;
    rc = bq_aesc_plan(g, edges_uv, k, eps, 0.0, BQ_PLAN_SCHEDULED, &tau_only, tau, nwalks);
    if (rc || k == 0) return rc;
    for (uint64_t q = 0; q < k; ++q)
        if (2ull * n_pilot * tau[q] >= (1ull << 32))
            return fail(BQ_EOVERFLOW, "query %llu: 2 * n_pilot * tau reaches 2^32", (unsigned long long)q);
    // explicit pairs (canonical order when edges_uv is NULL)
    std::vector<uint32_t> canon;
    if (!edges_uv && !canonical_pairs_host(g, canon)) return fail(BQ_EGRAPH, "graph is not symmetric");
    const uint32_t *pairs = edges_uv ? edges_uv : canon.data();
    std::vector<uint32_t> n0(k, n_pilot);
    DeviceGuard guard(g->device);
    uint32_t *status = nullptr;
    rc = status_word(g->device, &status);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t eb = sizeof(uint32_t) * 2 * k, tb = sizeof(uint32_t) * k, mb = sizeof(uint64_t) * 10 * k;
    char *buf = nullptr;
    rc = scratch_alloc((void **)&buf, mb + eb + 3 * tb, s);
    if (rc) return rc;
    uint64_t *d_mo = (uint64_t *)buf;
    uint32_t *d_uv = (uint32_t *)(buf + mb);
    uint32_t *d_tau = (uint32_t *)(buf + mb + eb);
    uint32_t *d_n0 = (uint32_t *)(buf + mb + eb + tb);
    uint32_t *d_nw = (uint32_t *)(buf + mb + eb + 2 * tb);
    cudaError_t e = cudaMemcpyAsync(d_uv, pairs, eb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_tau, tau, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_n0, n0.data(), tb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "pilot upload");
    const PilotParams pp{n_pilot, sched->n_min, eps, z};
    if (rc == BQ_OK)
        rc = launch_aesc_moments(g->view(), seed, d_uv, k, d_tau, d_n0, smp, d_mo, &pp, d_nw, status, s);
    if (rc == BQ_OK) {
        e = cudaMemcpyAsync(nwalks, d_nw, tb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && moments) e = cudaMemcpyAsync(moments, d_mo, mb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "pilot download");
    }
    scratch_free(buf, s);
    if (rc == BQ_OK) rc = bq_sync(stream);
    else cudaStreamSynchronize(s);
    return rc;
}

int bq_aesc_estimate(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev, uint64_t k,
                     const uint32_t *tau_dev, const uint32_t *nwalks_dev, const bq_sampler *sampler, uint32_t flags,
                     uint32_t *counts_dev, double *sc_dev, void *stream) {
    bq::NvtxRange nvtx_range("bq_aesc_estimate");
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (flags & ~(BQ_HOST_IO | BQ_AESC_NAIVE)) return fail(BQ_EINVAL, "unknown AESC flags 0x%x", flags);
    const bool naive = (flags & BQ_AESC_NAIVE) != 0;
    if (k && (!tau_dev || !nwalks_dev || !counts_dev || !sc_dev))
        return fail(BQ_EINVAL, "tau, nwalks, counts or sc is NULL");
    if (!edges_uv_dev && (k != g->nnz / 2 || k != g->m_upper))
        return fail(BQ_EINVAL, "all-edges estimate needs k = m = %llu (got %llu; %llu edges above the diagonal)",
                    (unsigned long long)(g->nnz / 2), (unsigned long long)k, (unsigned long long)g->m_upper);
    Sampler smp;
    int rc = check_sampler(sampler, smp);
    if (rc) return rc;
    if (k == 0) return BQ_OK;
    DeviceGuard guard(g->device);
    uint32_t *status = nullptr;
    rc = status_word(g->device, &status);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!(flags & BQ_HOST_IO))
        return launch_aesc(g->view(), seed, edges_uv_dev, k, tau_dev, nwalks_dev, smp, naive, counts_dev, sc_dev,
                           status, s);

    const size_t eb = edges_uv_dev ? sizeof(uint32_t) * 2 * k : 0;
    const size_t tb = sizeof(uint32_t) * k, cb = sizeof(uint32_t) * 4 * k, scb = sizeof(double) * k;
    char *buf = nullptr;
    rc = scratch_alloc((void **)&buf, scb + cb + 2 * tb + eb, s);
    if (rc) return rc;
    double *d_sc = (double *)buf;
    uint32_t *d_counts = (uint32_t *)(buf + scb);
    uint32_t *d_tau = (uint32_t *)(buf + scb + cb);
    uint32_t *d_nw = (uint32_t *)(buf + scb + cb + tb);
    uint32_t *d_uv = edges_uv_dev ? (uint32_t *)(buf + scb + cb + 2 * tb) : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_tau, tau_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_nw, nwalks_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d_uv) e = cudaMemcpyAsync(d_uv, edges_uv_dev, eb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "host-io upload");
    if (rc == BQ_OK) rc = launch_aesc(g->view(), seed, d_uv, k, d_tau, d_nw, smp, naive, d_counts, d_sc, status, s);
    if (rc == BQ_OK) {
        e = cudaMemcpyAsync(counts_dev, d_counts, cb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc_dev, d_sc, scb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "host-io download");
    }
    scratch_free(buf, s);
    if (rc == BQ_OK) rc = bq_sync(stream);
    else cudaStreamSynchronize(s);
    return rc;
}

int bq_aesc_estimate_push(const bq_graph *g, uint64_t seed, const uint32_t *edges_uv_dev, uint64_t k,
                          const uint32_t *tau_dev, const uint32_t *nwalks_dev, uint32_t push_max,
                          uint32_t support_cap, uint32_t flags, uint32_t *depth_dev, uint64_t *acc_dev,
                          double *sc_dev, void *stream) {
    bq::NvtxRange nvtx_range("bq_aesc_estimate_push");
    g_last_error[0] = 0;
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (flags & ~BQ_HOST_IO) return fail(BQ_EINVAL, "unknown AESC flags 0x%x", flags);
    if (push_max > 8) return fail(BQ_EINVAL, "push_max = %u (at most 8)", push_max);
    if (support_cap == 0 || support_cap > kPushSupportCapMax)
        return fail(BQ_EINVAL, "support_cap = %u (1..%u: the pushed-vector tables hold %u vertices per side)",
                    support_cap, kPushSupportCapMax, kPushSupportCapMax);
    if (k && (!tau_dev || !nwalks_dev || !acc_dev || !sc_dev))
        return fail(BQ_EINVAL, "tau, nwalks, acc or sc is NULL");
    if (!edges_uv_dev && (k != g->nnz / 2 || k != g->m_upper))
        return fail(BQ_EINVAL, "all-edges estimate needs k = m = %llu (got %llu; %llu edges above the diagonal)",
                    (unsigned long long)(g->nnz / 2), (unsigned long long)k, (unsigned long long)g->m_upper);
    if (k == 0) return BQ_OK;
    DeviceGuard guard(g->device);
    uint32_t *status = nullptr;
    int rc = status_word(g->device, &status);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!(flags & BQ_HOST_IO))
        return launch_aesc_push(g->view(), seed, edges_uv_dev, k, tau_dev, nwalks_dev, push_max, support_cap,
                                depth_dev, acc_dev,
                                sc_dev, status, s);

    const size_t eb = edges_uv_dev ? sizeof(uint32_t) * 2 * k : 0;
    const size_t tb = sizeof(uint32_t) * k, ab = sizeof(uint64_t) * 4 * k, scb = sizeof(double) * k;
    char *buf = nullptr;
    rc = scratch_alloc((void **)&buf, scb + ab + 3 * tb + eb, s);
    if (rc) return rc;
    double *d_sc = (double *)buf;
    uint64_t *d_acc = (uint64_t *)(buf + scb);
    uint32_t *d_tau = (uint32_t *)(buf + scb + ab);
    uint32_t *d_nw = (uint32_t *)(buf + scb + ab + tb);
    uint32_t *d_depth = (uint32_t *)(buf + scb + ab + 2 * tb);
    uint32_t *d_uv = edges_uv_dev ? (uint32_t *)(buf + scb + ab + 3 * tb) : nullptr;
    cudaError_t e = cudaMemcpyAsync(d_tau, tau_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_nw, nwalks_dev, tb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && d_uv) e = cudaMemcpyAsync(d_uv, edges_uv_dev, eb, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "host-io upload");
    if (rc == BQ_OK)
        rc = launch_aesc_push(g->view(), seed, d_uv, k, d_tau, d_nw, push_max, support_cap, d_depth, d_acc, d_sc,
                              status, s);
    if (rc == BQ_OK) {
        e = cudaMemcpyAsync(acc_dev, d_acc, ab, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sc_dev, d_sc, scb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && depth_dev) e = cudaMemcpyAsync(depth_dev, d_depth, tb, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) rc = cuda_fail(e, "host-io download");
    }
    scratch_free(buf, s);
    if (rc == BQ_OK) rc = bq_sync(stream);
    else cudaStreamSynchronize(s);
    return rc;
}

int bq_sync(void *stream) {
    g_last_error[0] = 0;
    cudaStream_t s = (cudaStream_t)stream;
    BQ_CUDA(cudaStreamSynchronize(s));
    int dev = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    uint32_t *status = nullptr;
    int rc = status_word(dev, &status);
    if (rc) return rc;
    uint32_t bits = 0;
    BQ_CUDA(cudaMemcpy(&bits, status, sizeof(bits), cudaMemcpyDeviceToHost));
    if (!bits) return BQ_OK;
    BQ_CUDA(cudaMemset(status, 0, sizeof(uint32_t)));
    if (bits & kStatusBadStart) return fail(BQ_EINVAL, "a walk start id was >= n (those walks were skipped)");
    if (bits & kStatusNoEdge) return fail(BQ_ENOEDGE, "a queried pair is not an edge (its estimate is NaN)");
    if (bits & kStatusOverflow) return fail(BQ_EOVERFLOW, "a uint32 counter wrapped or 2 N tau >= 2^32");
    if (bits & kStatusBadIndex) return fail(BQ_EINVAL, "a query had tau = 0 or nwalks = 0 (its estimate is NaN)");
    if (bits & kStatusTimeout) return fail(BQ_ETIMEOUT, "a bounded device wait gave up");
    if (bits & kStatusRepeated) return fail(BQ_EINVAL, "an edge was queried twice in a vertex-centric estimate");
    if (bits & kStatusPlanGrew)
        return fail(BQ_EINVAL, "a vertex-centric batch's plan needs longer return histograms than at its creation "
                               "(a vertex's largest tau grew; its estimates are NaN)");
    return fail(BQ_ECUDA, "unknown device status bits 0x%x", bits);
}

int bq_profile_enable(int enable) {
    g_prof_enabled.store(enable ? 1 : 0);
    return BQ_OK;
}

int bq_profile_read(bq_profile *out) {
    g_last_error[0] = 0;
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    std::vector<PendingTiming> pending;
    {
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        pending.swap(g_prof_pending);
    }
    int rc = BQ_OK;
    for (const PendingTiming &p : pending) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(p.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.start, p.stop);
        if (e != cudaSuccess && rc == BQ_OK) rc = cuda_fail(e, "bq_profile_read");
        std::lock_guard<std::mutex> lock(g_prof_mutex);
        g_prof_ms[p.kind] += ms;
        g_prof_count[p.kind] += 1;
        g_prof_free_events.push_back(p.start);
        g_prof_free_events.push_back(p.stop);
    }
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    out->walk_ms = g_prof_ms[kProfWalk];
    out->walk_launches = g_prof_count[kProfWalk];
    out->group_ms = g_prof_ms[kProfGroup];
    out->group_launches = g_prof_count[kProfGroup];
    out->aesc_ms = g_prof_ms[kProfAesc];
    out->aesc_launches = g_prof_count[kProfAesc];
    out->aesc_aux_ms = g_prof_ms[kProfAescAux];
    out->aesc_aux_launches = g_prof_count[kProfAescAux];
    out->kernel_launches = g_launches.exchange(0);
    for (int i = 0; i < 8; ++i) out->walk_kernel_launches[i] = g_walk_kernels[i].exchange(0);
    for (int i = 0; i < 4; ++i) {
        g_prof_ms[i] = 0.0;
        g_prof_count[i] = 0;
    }
    return rc;
}

int bq_get_tuning(bq_tuning *out) {
    if (!out) return fail(BQ_EINVAL, "out is NULL");
    memset(out, 0, sizeof(*out));
    out->walk_lanes = (uint32_t)g_walks_per_lane.load();
    out->aggregate_visits = (uint32_t)g_aggregate.load();
    out->aesc_lanes = (uint32_t)g_aesc_walks_per_lane.load();
    out->layout = (uint32_t)g_edge_records.load();
    out->hub_slots = (uint32_t)g_hub_slots.load();
    out->l2_hints = (uint32_t)g_l2_hints.load();
    out->aesc_hub = (uint32_t)g_aesc_hub.load();
    out->hub_cluster = (uint32_t)g_hub_cluster.load();
    out->hub_relabel = (uint32_t)g_hub_relabel.load();
    out->relabel_hub8 = (uint32_t)g_relabel_hub8.load();
    out->hub8_hubs = (uint32_t)g_hub8_hubs.load();
    out->hub8_count_bits = (uint32_t)g_hub8_count_bits.load();
    out->shared_lanes = (uint32_t)g_shared_lanes.load();
    out->group_walks = (uint32_t)g_group_walks.load();
    out->push_lanes = (uint32_t)g_push_lanes.load();
    return BQ_OK;
}

int bq_set_tuning(const bq_tuning *in) {
    g_last_error[0] = 0;
    if (!in) return fail(BQ_EINVAL, "tuning is NULL");
    const uint32_t w = in->walk_lanes, a = in->aesc_lanes;
    if (w != 1 && w != 2 && w != 4 && w != 8) return fail(BQ_EINVAL, "walk_lanes must be 1, 2, 4 or 8");
    if (a != 2 && a != 4 && a != 8) return fail(BQ_EINVAL, "aesc_lanes must be 2, 4 or 8");
    if (in->aggregate_visits > 1) return fail(BQ_EINVAL, "aggregate_visits must be 0 or 1");
    if (in->layout > 5) return fail(BQ_EINVAL, "layout must be 0 to 5");
    if (in->hub_slots != 0 && (in->hub_slots < 1024 || in->hub_slots > kHubSlotsMax))
        return fail(BQ_EINVAL, "hub_slots must be 0 or 1024..%u", kHubSlotsMax);
    if (in->l2_hints > 1) return fail(BQ_EINVAL, "l2_hints must be 0 or 1");
    if (in->aesc_hub > 1) return fail(BQ_EINVAL, "aesc_hub must be 0 or 1");
    const uint32_t c = in->hub_cluster;
    if (c != 0 && c != 1 && c != 2 && c != 4 && c != 8) return fail(BQ_EINVAL, "hub_cluster must be 0, 1, 2, 4 or 8");
    if (in->hub_relabel > 1) return fail(BQ_EINVAL, "hub_relabel must be 0 or 1");
    if (in->relabel_hub8 > 1) return fail(BQ_EINVAL, "relabel_hub8 must be 0 or 1");
    if (in->hub8_hubs > kHub8Max) return fail(BQ_EINVAL, "hub8_hubs must be at most %u", kHub8Max);
    if (in->hub8_count_bits > 31) return fail(BQ_EINVAL, "hub8_count_bits must be 0..31");
    if (in->shared_lanes != 2 && in->shared_lanes != 4 && in->shared_lanes != 8)
        return fail(BQ_EINVAL, "shared_lanes must be 2, 4 or 8");
    if (in->group_walks > 1) return fail(BQ_EINVAL, "group_walks must be 0 or 1");
    if (in->push_lanes != 2 && in->push_lanes != 4 && in->push_lanes != 8)
        return fail(BQ_EINVAL, "push_lanes must be 2, 4 or 8");
    g_walks_per_lane.store((int)w);
    g_aggregate.store((int)in->aggregate_visits);
    g_aesc_walks_per_lane.store((int)a);
    g_edge_records.store((int)in->layout);
    g_hub_slots.store((int)in->hub_slots);
    g_l2_hints.store((int)in->l2_hints);
    g_aesc_hub.store((int)in->aesc_hub);
    g_hub_cluster.store(c < 1 ? 1 : (int)c);
    g_hub_relabel.store((int)in->hub_relabel);
    g_relabel_hub8.store((int)in->relabel_hub8);
    g_hub8_hubs.store((int)in->hub8_hubs);
    g_hub8_count_bits.store((int)in->hub8_count_bits);
    g_shared_lanes.store((int)in->shared_lanes);
    g_group_walks.store((int)in->group_walks);
    g_push_lanes.store((int)in->push_lanes);
    return BQ_OK;
}

}  // extern "C"
