"""Vertex-centric AESC (walks shared by the query edges at a vertex) on the
GPU: counters, walk counts and FP64 estimates bit-identical to the oracle's
for both samplers, every layout, subsets and all edges, device tensors and
host buffers; errors."""

import numpy as np
import pytest

import oracle
from workloads import all_edges, chung_lu, er_with_path, gnp_connected, rmat

pytestmark = pytest.mark.gpu

SCHED = (2.0, 2, 64, 9.0, 32)


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def same_bits(a, b):
    return np.array_equal(np.asarray(a, np.float64).view(np.uint64), np.asarray(b, np.float64).view(np.uint64))


def check(bq, graph, g, seed, uv, tau, nw, sampler=None):
    counts, nused, sc = bq.aesc_estimate_shared_host(graph, seed, uv, tau, nw, sampler)
    q = uv if uv is not None else all_edges(g)
    oc, on, osc = oracle.aesc_shared_estimate(g, seed, q, tau, nw, sampler)
    assert np.array_equal(counts, oc)
    assert np.array_equal(nused, on)
    assert same_bits(sc, osc)
    return counts, nused, sc


@pytest.mark.parametrize("sampler", [None, (1, 8, 32)], ids=["ind", "coupled"])
def test_subset_bit_exact(env, sampler):
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(4)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    uv[::2] = uv[::2, ::-1]
    tau, nw = oracle.plan_scheduled(g, uv, 0.1, *SCHED)
    nw[::5] += 97  # ragged 128-walk tasks and unequal N at shared endpoints
    tau[::7] += 3
    _, nused, _ = check(bq, graph, g, 9, uv, tau, nw, sampler)
    assert np.any(nused.reshape(-1, 2) > nw[:, None])


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_layouts_never_change_results(env, layout):
    bq, torch = env
    g = rmat(12, 8, seed=5)
    rng = np.random.default_rng(2)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.1, *SCHED)
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        for lanes in (2, 4, 8):  # walks per lane: the task grouping, never a result
            bq.set_tuning(shared_lanes=lanes)
            check(bq, graph, g, 5, uv, tau, nw)
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_all_edges_ragged(env):
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    graph = bq.Graph.from_csr(g)
    k = all_edges(g).shape[0]
    tau = (np.arange(k, dtype=np.uint32) % 5) + 1
    nw = ((np.arange(k, dtype=np.uint32) * 53) % 700 + 1).astype(np.uint32)
    check(bq, graph, g, 13, None, tau, nw)


def test_device_tensors_match_host_buffers(env):
    bq, torch = env
    g = chung_lu(20000, 8.0, 2.2, 3)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(6)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 500, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.05, *SCHED)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    counts, nused, sc = bq.aesc_estimate_shared(graph, 77, dev(uv), dev(tau), dev(nw))
    bq.sync()
    c2, n2, s2 = check(bq, graph, g, 77, uv, tau, nw)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), c2)
    assert np.array_equal(nused.cpu().numpy().view(np.uint32), n2)
    assert same_bits(sc.cpu().numpy(), s2)


def test_power_law_all_edges_sampled(env):
    """All edges of a 200k-vertex power-law graph in one call.  An edge's
    result depends on the query edges at its two endpoints only, so the
    oracle runs on the edges at the endpoints of 200 sampled edges."""
    bq, torch = env
    g = chung_lu(200000, 10.0, 2.1, 8)
    graph = bq.Graph.from_csr(g)
    uv_all = all_edges(g)
    tau, nw = oracle.plan_scheduled(g, uv_all, 0.1, *SCHED)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    counts, nused, sc = bq.aesc_estimate_shared(graph, 3, None, dev(tau), dev(nw))
    bq.sync()
    counts = counts.cpu().numpy().view(np.uint32).reshape(-1, 4)
    nused = nused.cpu().numpy().view(np.uint32).reshape(-1, 2)
    sc = sc.cpu().numpy()
    rng = np.random.default_rng(1)
    low = np.maximum(g.degrees[uv_all[:, 0]], g.degrees[uv_all[:, 1]]) <= 40  # keep the oracle's sub-query small
    pick = rng.choice(np.flatnonzero(low), 200, replace=False)
    ends = np.unique(uv_all[pick].ravel())
    touch = np.flatnonzero(np.isin(uv_all[:, 0], ends) | np.isin(uv_all[:, 1], ends))
    oc, on, osc = oracle.aesc_shared_estimate(g, 3, uv_all[touch], tau[touch], nw[touch])
    where = {int(e): i for i, e in enumerate(touch)}
    rows = np.array([where[int(p)] for p in pick])
    assert np.array_equal(counts[pick], oc.reshape(-1, 4)[rows])
    assert np.array_equal(nused[pick], on.reshape(-1, 2)[rows])
    assert same_bits(sc[pick], osc[rows])
    assert np.all(np.isfinite(sc))


def test_errors(env):
    bq, torch = env
    g = gnp_connected(30, 0.2, 2)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)[:3]
    tau = np.full(3, 3, np.uint32)
    nw = np.full(3, 10, np.uint32)
    dup = np.concatenate([uv, uv[1:2, ::-1]])
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_shared_host(graph, 1, dup, np.full(4, 3, np.uint32), np.full(4, 10, np.uint32))
    assert ei.value.code == bq.EINVAL
    row0 = set(g.row(0).tolist())
    non = next(x for x in range(1, g.n) if x not in row0)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_shared_host(graph, 1, np.array([[0, non]], np.uint32), tau[:1], nw[:1])
    assert ei.value.code == bq.ENOEDGE
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_shared_host(graph, 1, uv, np.array([3, 0, 3], np.uint32), nw)
    assert ei.value.code == bq.EINVAL
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_shared_host(graph, 1, uv, np.full(3, 64, np.uint32), np.full(3, 1 << 25, np.uint32))
    assert ei.value.code == bq.EOVERFLOW
    # the context is still usable
    check(bq, graph, g, 2, uv, tau, nw)
