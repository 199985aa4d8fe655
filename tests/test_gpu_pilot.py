"""Pilot plan on the GPU: the pilot's moments, tau and walk counts
bit-identical to the oracle's for every sampler, layout and edge subset; the
pilot's walks are the estimate's first walks; errors and degenerate cases."""

import numpy as np
import pytest

import oracle
from workloads import all_edges, chung_lu, er_with_path, gnp_connected, path, rmat

pytestmark = pytest.mark.gpu

SCHED = (2.0, 2, 64, 9.0, 32)  # tau_scale, tau_add, tau_max, n_scale (unused), n_min


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def schedule(bq):
    return bq.Schedule(SCHED[0], SCHED[1], SCHED[2], SCHED[3], SCHED[4], 0)


def check(bq, graph, g, seed, uv, eps, n_pilot, z=3.0, sampler=None):
    tau, nw, mo = bq.aesc_plan_pilot(graph, seed, uv, eps, schedule(bq), n_pilot, z, sampler)
    q = uv if uv is not None else all_edges(g)
    ot, on, om, _ = oracle.plan_pilot(g, seed, q, eps, SCHED[0], SCHED[1], SCHED[2], SCHED[4], n_pilot, z,
                                      sampler)
    assert np.array_equal(tau, ot)
    assert np.array_equal(mo, om)
    assert np.array_equal(nw, on)
    return tau, nw, mo


@pytest.mark.parametrize("sampler", [None, (1, 8, 32), (1, 32, 4)], ids=["ind", "coupled8", "coupled32"])
def test_subset_bit_exact(env, sampler):
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(4)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    uv[::2] = uv[::2, ::-1]
    # 200 walks per side: three full 64-walk tasks and a ragged one
    _, nw, _ = check(bq, graph, g, 9, uv, 0.1, 200, sampler=sampler)
    assert nw.min() >= SCHED[4] and nw.max() > SCHED[4]


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_layouts_never_change_results(env, layout):
    bq, torch = env
    g = rmat(12, 8, seed=5)
    rng = np.random.default_rng(2)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 300, replace=False)]
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        check(bq, graph, g, 5, uv, 0.1, 130)
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_all_edges(env):
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    graph = bq.Graph.from_csr(g)
    tau, nw, _ = check(bq, graph, g, 13, None, 0.05, 64, z=2.0)
    t2, n2, mo = bq.aesc_plan_pilot(graph, 13, None, 0.05, schedule(bq), 64, 2.0, moments=False)
    assert mo is None and np.array_equal(t2, tau) and np.array_equal(n2, nw)


def test_pilot_walks_are_the_estimate_first_walks(env):
    """Sum a and sum b of each side are the counters of an estimate with
    N = n_pilot walks and the same tau."""
    bq, torch = env
    g = er_with_path(2000, 9000, 7)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)[::17]
    tau, _, mo = bq.aesc_plan_pilot(graph, 21, uv, 0.1, schedule(bq), 97)
    counts, _ = bq.aesc_estimate_host(graph, 21, uv, tau, np.full(uv.shape[0], 97, np.uint32))
    counts = counts.reshape(-1, 2, 2).astype(np.uint64)
    assert np.array_equal(mo[:, :, 0], counts[:, :, 0])
    assert np.array_equal(mo[:, :, 1], counts[:, :, 1])


def test_power_law_sampled_edges(env):
    """All edges of a 200k-vertex power-law graph in one pilot; 400 sampled
    edges against the oracle (an edge's walks depend only on its own id)."""
    bq, torch = env
    g = chung_lu(200000, 10.0, 2.1, 8)
    graph = bq.Graph.from_csr(g)
    uv_all = all_edges(g)
    tau, nw, mo = bq.aesc_plan_pilot(graph, 3, None, 0.05, schedule(bq), 64)
    idx = np.random.default_rng(1).choice(uv_all.shape[0], 400, replace=False)
    ot, on, om, _ = oracle.plan_pilot(g, 3, uv_all[idx], 0.05, SCHED[0], SCHED[1], SCHED[2], SCHED[4], 64)
    assert np.array_equal(tau[idx], ot)
    assert np.array_equal(mo[idx], om)
    assert np.array_equal(nw[idx], on)


def test_zero_variance_and_errors(env):
    bq, torch = env
    g = path(2)
    graph = bq.Graph.from_csr(g)
    tau, nw, mo = bq.aesc_plan_pilot(graph, 1, None, 0.05, bq.Schedule(2.0, 2, 64, 9.0, 17, 0), 50)
    assert nw[0] == 17
    g = gnp_connected(30, 0.2, 2)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)[:3]
    for n_pilot, z in ((1, 3.0), (10, 0.0)):
        with pytest.raises(bq.BouquetError) as ei:
            bq.aesc_plan_pilot(graph, 1, uv, 0.1, schedule(bq), n_pilot, z)
        assert ei.value.code == bq.EINVAL
    row0 = set(g.row(0).tolist())
    non = next(x for x in range(1, g.n) if x not in row0)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan_pilot(graph, 1, np.array([[0, non]], np.uint32), 0.1, schedule(bq), 10)
    assert ei.value.code == bq.ENOEDGE
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan_pilot(graph, 1, uv, 0.1, schedule(bq), 1 << 30)
    assert ei.value.code == bq.EOVERFLOW
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan_pilot(graph, 1, uv, 1e-7, schedule(bq), 100)
    assert ei.value.code == bq.EOVERFLOW
