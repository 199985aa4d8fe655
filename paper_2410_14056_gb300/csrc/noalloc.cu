// bq_walk_batch_noalloc: the bouquet walk batch for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc or any other allocator during a call:
// a plug-in running inside a host application that owns every byte of device
// memory, a latency-critical loop in which an allocation could block, fail
// or fragment at an arbitrary moment, or code running under a memory cap that
// has already been handed out in full.  The ordinary entry point takes its
// temporary buffers (the counting sort that groups walks by start vertex)
// from the stream-ordered pool; this one takes them from a fixed array in the
// library's own device memory instead, so a call allocates nothing.
//
// The array is a file-scope __device__ variable of kStaticScratchBytes.  Every
// device on which this module is loaded holds it until the process exits.  In
// host code its name is only a host-side stand-in, so the device address is
// looked up with cudaGetSymbolAddress once per device (on the first call made
// with that device current) and cached.  Because of that set-up, make the
// first call on each device before any stream capture.  All calls share the
// array and it keeps the last call's contents: the call clears what must
// start at zero, and calls whose work overlaps on the GPU (different streams,
// or graph launches in flight together) race on it.
#include <mutex>
#include <vector>

#include "internal.h"

namespace bq {
namespace {

constexpr size_t kStaticScratchBytes = 32ull << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_noalloc_mutex;
std::vector<void *> g_noalloc_ptr;  // per device ordinal, looked up once

int static_scratch_address(int device, void **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if ((int)g_noalloc_ptr.size() <= device) g_noalloc_ptr.resize(device + 1, nullptr);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static walk scratch)");
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return BQ_OK;
}

}  // namespace
}  // namespace bq

using namespace bq;

extern "C" int bq_walk_batch_noalloc(const bq_graph *g, uint64_t seed, const uint32_t *starts_dev, uint64_t n_walks,
                                     uint32_t n_steps, const bq_sampler *sampler, uint32_t flags,
                                     uint32_t *visits_dev, uint32_t *paths_dev, void *stream) {
    bq::NvtxRange nvtx_range("bq_walk_batch_noalloc");
    clear_error();
    if (!g) return fail(BQ_EINVAL, "graph is NULL");
    if (flags & ~BQ_VISIT_START)
        return fail(BQ_EINVAL, "bq_walk_batch_noalloc takes device buffers only (flags 0x%x)", flags);
    if (n_walks && (!starts_dev || !visits_dev)) return fail(BQ_EINVAL, "starts or visits is NULL");
    if (n_walks >= (1ull << 32)) return fail(BQ_EINVAL, "n_walks must be < 2^32");
    if (paths_dev && n_walks > UINT64_MAX / ((uint64_t)n_steps + 1) / sizeof(uint32_t))
        return fail(BQ_EINVAL, "paths array size overflows");
    Sampler smp;
    int rc = validate_sampler(sampler, smp, true);
    if (rc) return rc;
    if (n_walks == 0) return BQ_OK;  // nothing to run, whatever the graph's size
    const size_t need = walk_batch_scratch_bytes(g->n, n_walks);
    if (need > kStaticScratchBytes)
        return fail(BQ_EINVAL,
                    "bq_walk_batch_noalloc needs %zu bytes of scratch for n = %u and %llu walks; its static "
                    "scratch holds %zu bytes (use bq_walk_batch, or split the batch)",
                    need, g->n, (unsigned long long)n_walks, kStaticScratchBytes);
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != g->device) {
        cudaError_t e = cudaSetDevice(g->device);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    }
    uint32_t *status = nullptr;
    void *scratch = nullptr;
    rc = existing_status_word(g->device, &status);
    if (rc == BQ_OK) rc = static_scratch_address(g->device, &scratch);
    if (rc == BQ_OK)
        rc = launch_walk_batch_in(g->view(), seed, starts_dev, n_walks, n_steps, smp, (flags & BQ_VISIT_START) != 0,
                                  visits_dev, paths_dev, status, scratch, kStaticScratchBytes, (cudaStream_t)stream);
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return rc;
}
