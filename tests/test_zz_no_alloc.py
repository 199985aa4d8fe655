"""bq_walk_batch_noalloc against bq_walk_batch, through the C ABI.

Some callers of this library cannot allocate device memory during a call: a
plug-in whose host application owns all device memory, a latency-critical
loop where an allocation could block or fail at any moment, or code under a
memory cap that is already handed out.  bq_walk_batch_noalloc serves them
from a fixed device array inside the library.  These tests check that it
returns exactly what the ordinary bouquet walk batch returns (visit counts
and paths are integers: bit-exact), on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next call), and
that a batch too large for the array is refused with a clear error."""

import ctypes

import numpy as np
import pytest

from workloads import rmat, uniform_starts

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


def test_noalloc_refuses_batch_beyond_static_scratch(env):
    bq, torch = env
    g = rmat(14, 8, seed=31)
    graph = bq.Graph.from_csr(g)
    L = bq.load_library()
    n_walks = 1 << 23  # 4 * (2 n + 1 + 2 n_walks) bytes > 32 MiB
    st = torch.zeros(n_walks, dtype=torch.int32, device="cuda")
    vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    rc = L.bq_walk_batch_noalloc(graph.handle, 1, ptr(st), n_walks, 8, None, 0, ptr(vis), None,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bq.EINVAL
    msg = L.bq_last_error().decode()
    assert "static scratch holds" in msg and str(32 << 20) in msg
    assert int(vis.sum()) == 0
    graph.close()
