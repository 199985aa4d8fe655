"""The profiling calls (the paper has no counterpart): launch counts per walk
kernel and the read-bandwidth probe used for roofline ceilings."""

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


def test_walk_kernel_launch_counts(env):
    """Each walk batch counts one launch of the kernel that ran, by kind."""
    bq, torch = env
    g = rmat(12, 8, seed=2)
    st = torch.from_numpy(uniform_starts(g, 5000, 1).view(np.int32)).cuda()
    old = bq.get_tuning()
    try:
        cases = [(dict(hub_slots=0, layout=0), bq.MODE_BOUQUET, "bouquet"),
                 (dict(hub_slots=1024, layout=5), bq.MODE_BOUQUET, "hub"),
                 (dict(hub_slots=1024, layout=5, hub_relabel=1, relabel_hub8=0), bq.MODE_BOUQUET, "relabel"),
                 (dict(hub_slots=1024, layout=5, hub_relabel=1, relabel_hub8=1), bq.MODE_BOUQUET, "relabel8"),
                 (dict(hub_slots=0, layout=0), bq.MODE_NAIVE, "naive")]
        for tuning, mode, kind in cases:
            bq.set_tuning(**tuning)
            graph = bq.Graph.from_csr(g)
            bq.profile_read()
            bq.walk_batch(graph, 3, st, 9, mode=mode)
            bq.walk_batch(graph, 4, st, 9, mode=mode)
            bq.sync()
            counts = bq.profile_read()["walk_kernels"]
            assert counts[kind] == 2 and sum(counts.values()) == 2, (kind, counts)
            graph.close()
            bq.set_tuning(**old)
    finally:
        bq.set_tuning(**old)


def test_read_bandwidth_probe(env):
    bq, torch = env
    buf = torch.ones(4 << 20, dtype=torch.int32, device="cuda")  # 16 MiB, L2-resident
    gbs = bq.read_bandwidth(buf, 50)
    assert np.isfinite(gbs) and 100.0 < gbs < 100_000.0
    assert torch.equal(buf, torch.ones_like(buf))  # read only
    L = bq.load_library()
    out = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.bq_profile_read_bandwidth(ctypes.c_void_p(buf.data_ptr() + 4), 1024, 1, stream,
                                       ctypes.byref(out)) == bq.EINVAL
    assert L.bq_profile_read_bandwidth(ctypes.c_void_p(buf.data_ptr()), 8, 1, stream, ctypes.byref(out)) == bq.EINVAL
    assert L.bq_profile_read_bandwidth(ctypes.c_void_p(buf.data_ptr()), 1024, 0, stream,
                                       ctypes.byref(out)) == bq.EINVAL
