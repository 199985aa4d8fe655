"""bq_walk_batch_noalloc against bq_walk_batch and the oracle, through the C ABI.

Some callers of this library cannot allocate device memory during a call: a
plug-in whose host application owns all device memory, a latency-critical
loop where an allocation could block or fail at any moment, or code under a
memory cap that is already handed out.  bq_walk_batch_noalloc serves them
from a fixed device array inside the library.  These tests check that it
returns exactly what the ordinary bouquet walk batch returns (visit counts
and paths are integers: bit-exact), on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next call); that
it equals the CPU oracle on the degree-relabelled copy and on the
checked-counter path; that a call takes nothing from the device's
stream-ordered pool and no other device memory; and that a batch too large
for the array is refused with a clear error while an empty batch is not."""

import ctypes

import numpy as np
import pytest

import oracle
from workloads import csr_from_edges, rmat, uniform_starts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_noalloc_matches_ordinary_entry_point_twice(env):
    bq, torch = env
    g = rmat(14, 8, seed=31)
    graph = bq.Graph.from_csr(g)
    L = bq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, n_walks, n_steps) in enumerate([(101, 300001, 24), (202, 123457, 40)]):
        starts = uniform_starts(g, n_walks, 40 + call)
        st = torch.from_numpy(starts.view(np.int32)).cuda()
        ref_v = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        ref_p = torch.zeros((n_walks, n_steps + 1), dtype=torch.int32, device="cuda")
        na_v = torch.zeros_like(ref_v)
        na_p = torch.zeros_like(ref_p)
        rc = L.bq_walk_batch(graph.handle, seed, ptr(st), n_walks, n_steps, bq.MODE_BOUQUET, None,
                             bq.VISIT_START, ptr(ref_v), ptr(ref_p), stream)
        assert rc == bq.OK, L.bq_last_error()
        rc = L.bq_walk_batch_noalloc(graph.handle, seed, ptr(st), n_walks, n_steps, None,
                                     bq.VISIT_START, ptr(na_v), ptr(na_p), stream)
        assert rc == bq.OK, L.bq_last_error()
        assert L.bq_sync(stream) == bq.OK, L.bq_last_error()
        assert torch.equal(na_v, ref_v), f"visit counts differ on call {call}"
        assert torch.equal(na_p, ref_p), f"paths differ on call {call}"
        assert int(na_v.to(torch.int64).sum()) == n_walks * (n_steps + 1)
    graph.close()


def test_noalloc_relabelled_copy_matches_oracle_twice(env):
    """The kernel on the degree-relabelled copy runs from the static array
    too: visits and paths equal the oracle's on two calls in a row."""
    bq, torch = env
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=5, hub_relabel=1, hub_slots=1024)
        g = rmat(13, 8, seed=33)
        graph = bq.Graph.from_csr(g)
        info = graph.info()
        assert info["relabel_hubs"] > 0, "the relabelled copy was not built"
        L = bq.load_library()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        bq.profile_read()  # resets the launch counts
        for call, (seed, n_walks, n_steps) in enumerate([(7, 100003, 17), (8, 50021, 33)]):
            starts = uniform_starts(g, n_walks, 60 + call)
            want_v, want_p = oracle.walk_batch(g, seed, starts, n_steps, include_start=True, want_paths=True)
            st = torch.from_numpy(starts.view(np.int32)).cuda()
            vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
            paths = torch.zeros((n_walks, n_steps + 1), dtype=torch.int32, device="cuda")
            rc = L.bq_walk_batch_noalloc(graph.handle, seed, ptr(st), n_walks, n_steps, None,
                                         bq.VISIT_START, ptr(vis), ptr(paths), stream)
            assert rc == bq.OK, L.bq_last_error()
            assert L.bq_sync(stream) == bq.OK, L.bq_last_error()
            assert np.array_equal(host_u32(vis), want_v), f"visits differ from the oracle on call {call}"
            assert np.array_equal(host_u32(paths), want_p), f"paths differ from the oracle on call {call}"
        launched = bq.profile_read()["walk_kernels"]
        assert launched["relabel"] + launched["relabel8"] == 2, launched
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_noalloc_checked_counters_match_oracle(env):
    """More than 2^32 positions in one batch: the checked-counter path.
    Walks standing on isolated vertices stay put (n_steps + 1 visits each, a
    closed form); the few others are replayed by the oracle from their ids."""
    bq, torch = env
    g = csr_from_edges(9, [0, 1, 2, 5], [1, 2, 0, 6])  # 3, 4, 7, 8 isolated
    n_steps = 1 << 20
    n_walks = 4104  # n_walks * (n_steps + 1) > 2^32
    starts = np.array([3, 4, 7, 8] * 1024 + [0, 1, 2, 5, 6, 0, 5, 2], np.uint32)
    assert starts.size == n_walks
    live = np.flatnonzero(np.isin(starts, [0, 1, 2, 5, 6])).astype(np.uint64)
    want = np.zeros(g.n, np.int64)
    for v in (3, 4, 7, 8):
        want[v] = 1024 * (n_steps + 1)
    p = oracle.walk_paths_by_id(g, 77, live, starts[live.astype(np.int64)], n_steps)
    want += np.bincount(p.reshape(-1).astype(np.int64), minlength=g.n)
    assert want.max() < 2 ** 32
    graph = bq.Graph.from_csr(g)
    L = bq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = torch.from_numpy(starts.view(np.int32)).cuda()
    for call in range(2):
        vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        rc = L.bq_walk_batch_noalloc(graph.handle, 77, ptr(st), n_walks, n_steps, None, bq.VISIT_START,
                                     ptr(vis), None, stream)
        assert rc == bq.OK, L.bq_last_error()
        assert L.bq_sync(stream) == bq.OK, L.bq_last_error()
        assert np.array_equal(host_u32(vis).astype(np.int64), want), f"call {call}"
    # a counter that would pass 2^32 is reported
    vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    many = np.full(n_walks, 3, np.uint32)
    rc = L.bq_walk_batch_noalloc(graph.handle, 77, ptr(torch.from_numpy(many.view(np.int32)).cuda()), n_walks,
                                 n_steps, None, bq.VISIT_START, ptr(vis), None, stream)
    assert rc == bq.OK, L.bq_last_error()
    assert L.bq_sync(stream) == bq.EOVERFLOW
    graph.close()


def _default_pool(device):
    """The device's default stream-ordered pool, through the CUDA runtime the
    library itself loaded."""
    rt = ctypes.CDLL("libcudart.so.13")
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), device) == 0
    return rt, pool


USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent / UsedMemHigh


def test_noalloc_takes_no_device_memory(env):
    """Around two calls: the pool's high-water mark of used memory stays where
    it was, and the device's free memory does not change (no cudaMalloc)."""
    bq, torch = env
    g = rmat(14, 8, seed=31)
    graph = bq.Graph.from_csr(g)
    L = bq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n_walks, n_steps = 200003, 16
    st = torch.from_numpy(uniform_starts(g, n_walks, 9).view(np.int32)).cuda()
    vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    ref = torch.zeros_like(vis)
    assert L.bq_walk_batch(graph.handle, 5, ptr(st), n_walks, n_steps, bq.MODE_BOUQUET, None, 0, ptr(ref),
                           None, stream) == bq.OK
    # warm-up: kernels are loaded on first use
    assert L.bq_walk_batch_noalloc(graph.handle, 5, ptr(st), n_walks, n_steps, None, 0, ptr(vis), None,
                                   stream) == bq.OK
    assert L.bq_sync(stream) == bq.OK
    torch.cuda.synchronize()
    rt, pool = _default_pool(torch.cuda.current_device())
    cur = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_CURRENT, ctypes.byref(cur)) == 0
    assert rt.cudaMemPoolSetAttribute(pool, USED_MEM_HIGH, ctypes.byref(ctypes.c_uint64(0))) == 0
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        vis.zero_()
        assert L.bq_walk_batch_noalloc(graph.handle, 5, ptr(st), n_walks, n_steps, None, 0, ptr(vis), None,
                                       stream) == bq.OK, L.bq_last_error()
        assert L.bq_sync(stream) == bq.OK
        assert torch.equal(vis, ref)
    torch.cuda.synchronize()
    high = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, USED_MEM_HIGH, ctypes.byref(high)) == 0
    free1, _ = torch.cuda.mem_get_info()
    assert high.value <= cur.value, (high.value, cur.value)
    assert free1 == free0, (free0, free1)
    graph.close()


def test_noalloc_refuses_batch_beyond_static_scratch(env):
    bq, torch = env
    g = rmat(14, 8, seed=31)
    graph = bq.Graph.from_csr(g)
    L = bq.load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n_walks = 1 << 23  # beyond the 32 MiB array at any n
    st = torch.zeros(n_walks, dtype=torch.int32, device="cuda")
    vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    rc = L.bq_walk_batch_noalloc(graph.handle, 1, ptr(st), n_walks, 8, None, 0, ptr(vis), None, stream)
    assert rc == bq.EINVAL
    msg = L.bq_last_error().decode()
    assert "static scratch holds" in msg and str(32 << 20) in msg
    # a later call that succeeds leaves no stale message; an empty batch is
    # accepted without any size check
    rc = L.bq_walk_batch_noalloc(graph.handle, 1, ptr(st), 0, 8, None, 0, ptr(vis), None, stream)
    assert rc == bq.OK and L.bq_last_error().decode() == ""
    assert L.bq_sync(stream) == bq.OK
    assert int(vis.sum()) == 0
    graph.close()
