"""AESC with a push phase (depths 0 to 8) on the GPU: depths, fixed-point
accumulators and FP64 estimates bit-identical to the oracle's, for every
graph layout and lane count, through device tensors and host buffers."""

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


def check(bq, graph, g, seed, uv, tau, nw, push_max, cap=512):
    depth, acc, sc = bq.aesc_estimate_push_host(graph, seed, uv, tau, nw, push_max, support_cap=cap)
    od, oa, osc = oracle.aesc_push_estimate(g, seed, uv if uv is not None else all_edges(g), tau, nw, push_max,
                                            support_cap=cap)
    assert np.array_equal(depth, od)
    assert np.array_equal(acc, oa)
    assert same_bits(sc, osc)
    return depth


@pytest.mark.parametrize("push_max", [0, 1])
def test_subset_bit_exact_both_depths(env, push_max):
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(4)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    uv[::2] = uv[::2, ::-1]
    eps = np.where(np.arange(300) % 3 == 0, 0.05, 0.2)
    tau = np.zeros(300, np.uint32)
    nw = np.zeros(300, np.uint32)
    for e in (0.05, 0.2):
        sel = eps == e
        t, n = oracle.plan_scheduled(g, uv[sel], e, *SCHED)
        tau[sel], nw[sel] = t, n
    nw[::3] = 4  # 2N below d(u) + d(v): these edges stay at depth 0
    depth = check(bq, graph, g, 9, uv, tau, nw, push_max)
    if push_max:
        assert depth.any() and not depth.all()  # both depths in one launch
    else:
        assert not depth.any()


def test_all_edges_and_tau_one(env):
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    graph = bq.Graph.from_csr(g)
    k = all_edges(g).shape[0]
    tau = (np.arange(k, dtype=np.uint32) % 5) + 1  # includes tau = 1: depth-1 edges without walks
    nw = ((np.arange(k, dtype=np.uint32) * 53) % 700 + 1).astype(np.uint32)
    depth = check(bq, graph, g, 13, None, tau, nw, 1)
    assert np.any((depth == 1) & (tau == 1))


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_layouts_and_lanes_never_change_results(env, layout):
    bq, torch = env
    g = rmat(12, 8, seed=5)
    rng = np.random.default_rng(2)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 400, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.1, *SCHED)
    want = oracle.aesc_push_estimate(g, 5, uv, tau, nw, 1)
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        for lanes in (2, 4, 8):
            bq.set_tuning(push_lanes=lanes)
            depth, acc, sc = bq.aesc_estimate_push_host(graph, 5, uv, tau, nw, 1)
            assert np.array_equal(depth, want[0]) and np.array_equal(acc, want[1]) and same_bits(sc, want[2]), lanes
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_device_tensors_match_host_buffers(env):
    bq, torch = env
    g = chung_lu(20000, 8.0, 2.2, 3)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(6)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 500, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.05, *SCHED)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    depth, acc, sc = bq.aesc_estimate_push(graph, 77, dev(uv), dev(tau), dev(nw), 1)
    bq.sync()
    check(bq, graph, g, 77, uv, tau, nw, 1)
    d2, a2, s2 = bq.aesc_estimate_push_host(graph, 77, uv, tau, nw, 1)
    assert np.array_equal(depth.cpu().numpy().view(np.uint32), d2)
    assert np.array_equal(acc.cpu().numpy().view(np.uint64), a2)
    assert same_bits(sc.cpu().numpy(), s2)


def test_errors(env):
    bq, torch = env
    g = gnp_connected(30, 0.2, 2)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)[:3]
    tau = np.full(3, 3, np.uint32)
    nw = np.full(3, 10, np.uint32)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_push_host(graph, 1, uv, tau, nw, push_max=9)
    assert ei.value.code == bq.EINVAL
    for cap in (0, 513):  # the device tables hold 512 vertices per side and level
        with pytest.raises(bq.BouquetError) as ei:
            bq.aesc_estimate_push_host(graph, 1, uv, tau, nw, push_max=4, support_cap=cap)
        assert ei.value.code == bq.EINVAL and "support_cap" in str(ei.value)
    row0 = set(g.row(0).tolist())
    non = next(x for x in range(1, g.n) if x not in row0)
    bad = np.array([[0, non]], np.uint32)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_push_host(graph, 1, bad, tau[:1], nw[:1])
    assert ei.value.code == bq.ENOEDGE


# ------------------------------------------------------------ depths >= 2

@pytest.mark.parametrize("push_max", [2, 4, 8])
def test_deep_subset_bit_exact(env, push_max):
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(8)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    uv[::2] = uv[::2, ::-1]
    tau, nw = oracle.plan_scheduled(g, uv, 0.05, *SCHED)
    nw[::2] *= 6  # larger walk budgets: deeper pushes
    tau[::5] += 2
    depth = check(bq, graph, g, 21, uv, tau, nw, push_max)
    assert depth.max() >= 2 and np.any(depth <= 1)


def test_deep_all_edges_tau_at_depth(env):
    """All edges, tau from 1 to 5 and large budgets: edges pushed to their
    full tau run no walks."""
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    graph = bq.Graph.from_csr(g)
    k = all_edges(g).shape[0]
    tau = (np.arange(k, dtype=np.uint32) % 5) + 1
    nw = np.full(k, 40000, np.uint32)
    nw[::3] = 50
    depth = check(bq, graph, g, 13, None, tau, nw, 8)
    assert np.any((depth == tau) & (tau >= 2))


@pytest.mark.parametrize("layout", [0, 2, 4, 5])
def test_deep_layouts_and_lanes(env, layout):
    bq, torch = env
    g = rmat(12, 8, seed=5)
    rng = np.random.default_rng(2)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.05, *SCHED)
    nw *= 12
    want = oracle.aesc_push_estimate(g, 5, uv, tau, nw, 3)
    assert want[0].max() >= 2
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        for lanes in (2, 4, 8):
            bq.set_tuning(push_lanes=lanes)
            depth, acc, sc = bq.aesc_estimate_push_host(graph, 5, uv, tau, nw, 3)
            assert np.array_equal(depth, want[0]) and np.array_equal(acc, want[1]) and same_bits(sc, want[2]), lanes
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_deep_support_cap(env):
    """A 600-leaf star stops at depth 1; a 30 x 30 two-level tree stops where
    a level passes 512 vertices."""
    from workloads import csr_from_edges
    bq, torch = env
    star = csr_from_edges(601, np.zeros(600, np.int64), np.arange(1, 601), name="star600")
    uv = all_edges(star)[:40]
    graph = bq.Graph.from_csr(star)
    depth = check(bq, graph, star, 3, uv, np.full(40, 4, np.uint32), np.full(40, 20000, np.uint32), 4)
    assert np.all(depth == 1)
    u, v, nxt = [], [], 31
    for c in range(1, 31):
        u.append(0)
        v.append(c)
        for _ in range(30):
            u.append(c)
            v.append(nxt)
            nxt += 1
    tree = csr_from_edges(nxt, np.array(u), np.array(v), name="tree30x30")
    graph = bq.Graph.from_csr(tree)
    uv = all_edges(tree)
    check(bq, graph, tree, 4, uv, np.full(uv.shape[0], 5, np.uint32), np.full(uv.shape[0], 20000, np.uint32), 5)


def test_deep_device_tensors_and_power_law(env):
    bq, torch = env
    g = chung_lu(200000, 10.0, 2.1, 8)
    graph = bq.Graph.from_csr(g)
    uv_all = all_edges(g)
    tau, nw = oracle.plan_scheduled(g, uv_all, 0.05, *SCHED)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    depth, acc, sc = bq.aesc_estimate_push(graph, 3, None, dev(tau), dev(nw), 2)
    bq.sync()
    depth = depth.cpu().numpy().view(np.uint32)
    acc = acc.cpu().numpy().view(np.uint64).reshape(-1, 4)
    sc = sc.cpu().numpy()
    assert np.any(depth == 2) and np.all(np.isfinite(sc))
    rng = np.random.default_rng(1)
    pick = np.concatenate([rng.choice(np.flatnonzero(depth == 2), 200, replace=False),
                           rng.choice(np.flatnonzero(depth < 2), 100, replace=False)])
    od, oa, osc = oracle.aesc_push_estimate(g, 3, uv_all[pick], tau[pick], nw[pick], 2)
    assert np.array_equal(depth[pick], od)
    assert np.array_equal(acc[pick], oa.reshape(-1, 4))
    assert same_bits(sc[pick], osc)


@pytest.mark.parametrize("cap", [1, 8, 64, 200, 512])
def test_deep_support_cap_parameter(env, cap):
    """The support cap is a plan parameter both sides receive: depths,
    accumulators and estimates equal the oracle's for every cap, and a
    smaller cap never deepens a push."""
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(9)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    tau, nw = oracle.plan_scheduled(g, uv, 0.05, *SCHED)
    nw *= 10
    tau[::3] += 3
    depth = check(bq, graph, g, 31, uv, tau, nw, 8, cap)
    full = oracle.aesc_push_counts(g, 31, uv, tau, nw, 8, support_cap=512)[0]
    assert np.all(depth <= full)
    # on this workload caps up to 64 keep every edge at depth 1, 200 takes
    # 283 of the 300 edges to depth 2, 512 all of them
    assert (depth.max() >= 2) == (cap >= 200)
    assert (cap == 512) == np.array_equal(depth, full)
