// Autotuners: choose walks per lane (the GPU's bouquet width is 32 lanes x
// walks per lane) by timing the caller's own workload.  The choice changes
// speed only: every result is identical for every setting.
#include "internal.h"

using namespace bq;

namespace {

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

template <typename Run>
int time_once(Run &&run, cudaStream_t s, float *ms) {
    Events ev;
    BQ_CUDA(cudaEventCreate(&ev.a));
    BQ_CUDA(cudaEventCreate(&ev.b));
    int rc = run();  // warm-up
    if (rc) return rc;
    BQ_CUDA(cudaEventRecord(ev.a, s));
    rc = run();
    if (rc) return rc;
    BQ_CUDA(cudaEventRecord(ev.b, s));
    BQ_CUDA(cudaEventSynchronize(ev.b));
    BQ_CUDA(cudaEventElapsedTime(ms, ev.a, ev.b));
    return BQ_OK;
}

// Read bandwidth probe: a persistent grid (SMs x 2 blocks of 1024 threads)
// reads `words` 16-byte words `reps` times with coalesced vector loads and
// folds them into one xor per thread, written only if it equals a value the
// data cannot produce (so the loads are not removed).
__global__ void __launch_bounds__(1024) read_probe_kernel(const uint4 *__restrict__ buf, uint64_t words,
                                                          uint32_t reps, uint32_t *sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t r = 0; r < reps; ++r)
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += stride) {
            const uint4 v = __ldcg(buf + i);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9E3779B9u) *sink = acc;
}

}  // namespace

extern "C" {

int bq_profile_read_bandwidth(const void *buf_dev, uint64_t bytes, uint32_t reps, void *stream, double *gbs) {
    bq::NvtxRange nvtx_range("bq_profile_read_bandwidth");
    clear_error();
    if (!buf_dev || !gbs || bytes < 16 || reps == 0) return fail(BQ_EINVAL, "buffer, size, reps or gbs invalid");
    if (((uintptr_t)buf_dev & 15) != 0) return fail(BQ_EINVAL, "the buffer must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    BQ_CUDA(cudaGetDevice(&dev));
    BQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t *sink = nullptr;  // written only if a thread's fold equals the magic value
    int rc = scratch_alloc((void **)&sink, 16, s);
    if (rc) return rc;
    const uint64_t words = bytes / 16;
    auto run = [&]() {
        count_launches(1);
        read_probe_kernel<<<2 * sms, 1024, 0, s>>>((const uint4 *)buf_dev, words, reps, sink);
        return cudaGetLastError() == cudaSuccess ? BQ_OK : fail(BQ_ECUDA, "read_probe_kernel launch failed");
    };
    float ms = 0.f;
    rc = time_once(run, s, &ms);
    scratch_free(sink, s);
    if (rc) return rc;
    *gbs = (double)words * 16.0 * reps / (ms / 1e3) / 1e9;
    return BQ_OK;
}

int bq_autotune_walks(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev, uint64_t n_walks,
                      uint32_t n_steps, uint32_t *visits_dev, void *stream, uint32_t *best, float *ms) {
    bq::NvtxRange nvtx_range("bq_autotune_walks");
    if (!g || !best) return fail(BQ_EINVAL, "graph or best is NULL");
    bq_tuning saved;
    bq_get_tuning(&saved);
    const uint32_t candidates[3] = {1, 2, 4};
    float t[3] = {0, 0, 0};
    int rc = BQ_OK;
    for (int i = 0; i < 3 && rc == BQ_OK; ++i) {
        bq_tuning cur = saved;
        cur.walk_lanes = candidates[i];
        rc = bq_set_tuning(&cur);
        if (rc) break;
        rc = time_once(
            [&]() {
                return bq_walk_batch(g, seed, starts_dev, n_walks, n_steps, BQ_MODE_BOUQUET, nullptr, 0, visits_dev,
                                     nullptr, stream);
            },
            (cudaStream_t)stream, &t[i]);
    }
    if (rc == BQ_OK) rc = bq_sync(stream);
    if (rc) {
        bq_set_tuning(&saved);
        return rc;
    }
    int pick = 0;
    for (int i = 1; i < 3; ++i)
        if (t[i] < t[pick]) pick = i;
    saved.walk_lanes = candidates[pick];
    bq_set_tuning(&saved);
    *best = candidates[pick];
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = t[i];
    return BQ_OK;
}

int bq_autotune_aesc(const bq_aesc_query *queries, uint32_t n_queries, const bq_sampler *sampler, void *stream,
                     uint32_t *best, float *ms) {
    bq::NvtxRange nvtx_range("bq_autotune_aesc");
    if (!best) return fail(BQ_EINVAL, "best is NULL");
    bq_tuning saved;
    bq_get_tuning(&saved);
    const uint32_t candidates[3] = {2, 4, 8};
    float t[3] = {0, 0, 0};
    int rc = BQ_OK;
    for (int i = 0; i < 3 && rc == BQ_OK; ++i) {
        bq_tuning cur = saved;
        cur.aesc_lanes = candidates[i];
        rc = bq_set_tuning(&cur);
        if (rc) break;
        bq_batch *b = nullptr;
        rc = bq_batch_create(queries, n_queries, sampler, &b);  // reads aesc_lanes
        if (rc) break;
        rc = time_once([&]() { return bq_batch_run(b, stream); }, (cudaStream_t)stream, &t[i]);
        bq_batch_destroy(b);
    }
    if (rc == BQ_OK) rc = bq_sync(stream);
    if (rc) {
        bq_set_tuning(&saved);
        return rc;
    }
    int pick = 0;
    for (int i = 1; i < 3; ++i)
        if (t[i] < t[pick]) pick = i;
    saved.aesc_lanes = candidates[pick];
    bq_set_tuning(&saved);
    *best = candidates[pick];
    if (ms)
        for (int i = 0; i < 3; ++i) ms[i] = t[i];
    return BQ_OK;
}

}  // extern "C"
