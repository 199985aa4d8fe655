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

}  // namespace

extern "C" {

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
