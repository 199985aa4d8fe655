"""Graph store through the C ABI: validation failures are rejected with
BQ_EGRAPH and a message, info reports the structure, device/borrowed inputs
work."""

import numpy as np
import pytest

from workloads import csr_from_edges, cycle, gnp_connected, prufer_tree, rmat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def bad(bq, n, offsets, nbrs, match, flags=0):
    with pytest.raises(bq.BouquetError) as ei:
        bq.Graph(n, np.asarray(offsets, np.int64), np.asarray(nbrs, np.uint32), flags)
    assert ei.value.code == bq.EGRAPH, str(ei.value)
    assert match in str(ei.value), str(ei.value)


def test_validation_rejects(env):
    bq, _ = env
    bad(bq, 3, [1, 2, 3, 4], [1, 0, 0, 0], "offsets[0]")
    bad(bq, 3, [0, 2, 1, 4], [1, 2, 0, 0], "decrease")
    bad(bq, 2, [0, 1, 2], [5, 0], "id >= n")
    bad(bq, 2, [0, 1, 2], [0, 1], "self-loop")
    bad(bq, 3, [0, 2, 3, 4], [2, 1, 0, 0], "not strictly increasing")
    bad(bq, 3, [0, 2, 3, 4], [1, 1, 0, 0], "not strictly increasing")  # duplicate
    bad(bq, 3, [0, 1, 2, 2], [1, 2], "asymmetric")
    bad(bq, 3, [0, 1, 1, 1], [1], "odd")


def test_skip_validate_and_require_connected(env):
    bq, _ = env
    # asymmetric but in-bounds: accepted with SKIP_VALIDATE
    g = bq.Graph(3, np.array([0, 1, 2, 2], np.int64), np.array([1, 2], np.uint32), bq.SKIP_VALIDATE)
    g.close()
    two = csr_from_edges(4, [0, 2], [1, 3])
    with pytest.raises(bq.BouquetError) as ei:
        bq.Graph.from_csr(two, bq.REQUIRE_CONNECTED)
    assert "2 connected components" in str(ei.value)
    bq.Graph.from_csr(cycle(6), bq.REQUIRE_CONNECTED).close()


def test_info(env):
    bq, _ = env
    g = gnp_connected(60, 0.1, 1)
    info = bq.Graph.from_csr(g).info()
    assert info["n"] == 60 and info["m"] == g.m and info["nnz"] == g.nnz
    assert info["min_degree"] == g.degrees.min() and info["max_degree"] == g.degrees.max()
    assert info["n_components"] == 1 and info["bipartite"] == 0
    t = bq.Graph.from_csr(prufer_tree(12, 2)).info()
    assert t["bipartite"] == 1 and t["m"] == 11
    c = bq.Graph.from_csr(csr_from_edges(5, [0], [1])).info()
    assert c["n_components"] == 4 and c["min_degree"] == 0


def test_device_and_borrowed_inputs(env):
    bq, torch = env
    import oracle
    from workloads import uniform_starts
    g = rmat(11, 8, seed=7)
    off = torch.from_numpy(g.offsets).cuda()
    nb = torch.from_numpy(g.nbrs.view(np.int32)).cuda()
    starts = uniform_starts(g, 4000, 2)
    want = oracle.walk_batch(g, 4, starts, 10)
    for flags in (bq.DEVICE_PTRS, bq.DEVICE_PTRS | bq.BORROW):
        graph = bq.Graph(g.n, off, nb, flags)
        vis = bq.walk_batch_host(graph, 4, starts, 10)
        assert np.array_equal(vis, want)
        graph.close()


def test_empty_graph_and_empty_batch(env):
    bq, torch = env
    graph = bq.Graph(4, np.zeros(5, np.int64), np.zeros(0, np.uint32))
    assert graph.info()["m"] == 0
    vis = bq.walk_batch_host(graph, 1, np.array([0, 3], np.uint32), 5)
    assert vis.tolist() == [5, 0, 0, 5]
    assert bq.walk_batch_host(graph, 1, np.zeros(0, np.uint32), 5).sum() == 0
