"""AESC parity: GPU counters and FP64 estimates against the CPU oracle, bit
for bit, through the C ABI; the library's planner against the oracle's; and
the eps contract against exact spanning centrality."""

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import all_edges, complete, cycle, diamond, er_with_path, gnp_connected, prufer_tree

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


EXACT = [("K8", complete(8), 0.1), ("C10", cycle(10), 0.1), ("tree12", prufer_tree(12, 2), 0.2),
         ("gnp10", gnp_connected(10, 0.5, 3), 0.1), ("diamond", diamond(), 0.05)]


def loaded(bq, g):
    graph = bq.Graph.from_csr(g)
    _, l2, lneg = exact.spectrum(g)
    graph.set_spectrum(l2, lneg)
    return graph, l2, lneg


def same_bits(a, b):
    return np.array_equal(np.asarray(a, np.float64).view(np.uint64), np.asarray(b, np.float64).view(np.uint64))


@pytest.mark.parametrize("name,g,eps", EXACT, ids=[e[0] for e in EXACT])
def test_exact_cases_bit_exact_and_within_eps(env, name, g, eps):
    bq, torch = env
    graph, l2, lneg = loaded(bq, g)
    uv = all_edges(g)
    tau, nw = bq.aesc_plan(graph, uv, eps, 0.01)
    otau, onw = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
    assert np.array_equal(tau, otau) and np.array_equal(nw, onw)
    counts, sc = bq.aesc_estimate_host(graph, 11, uv, tau, nw)
    ocounts, osc = oracle.aesc_estimate(g, 11, uv, tau, nw)
    assert np.array_equal(counts, ocounts)
    assert same_bits(sc, osc)
    assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= eps


def test_tiny_aesc_workload(env):
    """ER n=1000, m=5000 plus a spanning path, all edges, certified eps=0.1:
    every estimate within eps of the pseudoinverse value; a 300-edge subset
    bit-exact against the oracle; subset results equal all-edges results."""
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph, l2, lneg = loaded(bq, g)
    uv = all_edges(g)
    tau, nw = bq.aesc_plan(graph, None, 0.1, 0.01)
    otau, onw = oracle.plan_certified(g, uv, 0.1, 0.01, l2, lneg)
    assert np.array_equal(tau, otau) and np.array_equal(nw, onw)
    counts, sc = bq.aesc_estimate(graph, 5, None, torch.from_numpy(tau.view(np.int32)).cuda(),
                                  torch.from_numpy(nw.view(np.int32)).cuda())
    bq.sync()
    counts = counts.cpu().numpy().view(np.uint32)
    sc = sc.cpu().numpy()
    assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= 0.1
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(uv.shape[0], 300, replace=False))
    ocounts, osc = oracle.aesc_estimate(g, 5, uv[pick], tau[pick], nw[pick])
    assert np.array_equal(counts.reshape(-1, 4)[pick].ravel(), ocounts)
    assert same_bits(sc[pick], osc)
    # the same pairs queried on their own, reversed: identical
    c2, s2 = bq.aesc_estimate_host(graph, 5, uv[pick][:, ::-1], tau[pick], nw[pick])
    assert np.array_equal(c2, ocounts) and same_bits(s2, osc)


@pytest.mark.parametrize("sampler", [(1, 4, 32), (1, 32, 8), (1, 0, 3)])
def test_coupled_sampler_bit_exact(env, sampler):
    bq, torch = env
    g = gnp_connected(30, 0.2, 4)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)
    tau = np.full(uv.shape[0], 7, np.uint32)
    nw = (np.arange(uv.shape[0], dtype=np.uint32) * 37) % 700 + 1
    counts, sc = bq.aesc_estimate_host(graph, 3, uv, tau, nw, sampler=sampler)
    ocounts, osc = oracle.aesc_estimate(g, 3, uv, tau, nw, sampler=sampler)
    assert np.array_equal(counts, ocounts) and same_bits(sc, osc)


def test_tuning_never_changes_results(env):
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)
    tau = (np.arange(uv.shape[0], dtype=np.uint32) % 9) + 1
    nw = (np.arange(uv.shape[0], dtype=np.uint32) * 53) % 1500 + 1
    want = oracle.aesc_counts(g, 9, uv, tau, nw)
    old = bq.get_tuning()
    try:
        for lanes in (2, 4, 8):
            bq.set_tuning(aesc_lanes=lanes)
            counts, _ = bq.aesc_estimate_host(graph, 9, uv, tau, nw)
            assert np.array_equal(counts, want), lanes
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_every_graph_layout_bit_exact(env, layout):
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    uv = all_edges(g)
    tau = (np.arange(uv.shape[0], dtype=np.uint32) % 9) + 1
    nw = (np.arange(uv.shape[0], dtype=np.uint32) * 53) % 1500 + 1
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        for sampler in (None, (1, 6, 32)):
            counts, sc = bq.aesc_estimate_host(graph, 13, uv, tau, nw, sampler=sampler)
            ocounts, osc = oracle.aesc_estimate(g, 13, uv, tau, nw, sampler=sampler)
            assert np.array_equal(counts, ocounts) and same_bits(sc, osc), sampler
        graph.close()
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("layout", [0, 5, 2])
def test_hub_table_never_changes_results(env, layout):
    """The hub variant of the counting kernel (hub records from shared
    memory) on a skewed graph where only part of the steps land on hubs, for
    several table sizes, both samplers, equal to the oracle and to the plain
    kernel."""
    bq, torch = env
    from workloads import rmat
    g = rmat(12, 8, seed=5)
    rng = np.random.default_rng(8)
    uv_all = all_edges(g)
    uv = uv_all[rng.choice(uv_all.shape[0], 700, replace=False)]
    tau = rng.integers(1, 12, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 900, uv.shape[0]).astype(np.uint32)
    old = bq.get_tuning()
    try:
        for hub_slots in (0, 1024, 5000, 13312):
            bq.set_tuning(layout=layout, hub_slots=hub_slots)
            graph = bq.Graph.from_csr(g)
            for sampler in (None, (1, 4, 32)):
                want = oracle.aesc_estimate(g, 21, uv, tau, nw, sampler=sampler)
                for hub in (1, 0):
                    bq.set_tuning(aesc_hub=hub)
                    counts, sc = bq.aesc_estimate_host(graph, 21, uv, tau, nw, sampler=sampler)
                    assert np.array_equal(counts, want[0]) and same_bits(sc, want[1]), (hub_slots, sampler, hub)
            graph.close()
    finally:
        bq.set_tuning(**old)


SCHEDULE = (2.0, 2, 64, 9.0, 32)  # tau_scale, tau_add, tau_max, n_scale, n_min (as the bench)


def test_scheduled_plan_matches_oracle(env):
    bq, torch = env
    from workloads import chung_lu
    for g in (er_with_path(1000, 5000, 1), chung_lu(20000, 10, 2.1, seed=5)):
        graph = bq.Graph.from_csr(g)
        uv = all_edges(g)
        sched = bq.Schedule(SCHEDULE[0], SCHEDULE[1], SCHEDULE[2], SCHEDULE[3], SCHEDULE[4], 0)
        tau, nw = bq.aesc_plan(graph, uv, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
        otau, onw = oracle.plan_scheduled(g, uv, 0.05, *SCHEDULE)
        assert np.array_equal(tau, otau) and np.array_equal(nw, onw)
        tau2, nw2 = bq.aesc_plan(graph, None, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
        assert np.array_equal(tau2, tau) and np.array_equal(nw2, nw)
        graph.close()


def test_large_plan_on_host_threads(env):
    """Plans of about 1M edges run on host threads: the same arrays as the
    oracle's, for a subset and for all edges, and of two bad pairs the lower
    index is the one reported."""
    bq, torch = env
    from workloads import chung_lu
    g = chung_lu(200000, 10.0, 2.1, 8)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)
    sched = bq.Schedule(SCHEDULE[0], SCHEDULE[1], SCHEDULE[2], SCHEDULE[3], SCHEDULE[4], 0)
    otau, onw = oracle.plan_scheduled(g, uv, 0.05, *SCHEDULE)
    tau, nw = bq.aesc_plan(graph, None, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    assert np.array_equal(tau, otau) and np.array_equal(nw, onw)
    rev = np.ascontiguousarray(uv[::-1, ::-1])
    tau, nw = bq.aesc_plan(graph, rev, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    assert np.array_equal(tau, otau[::-1]) and np.array_equal(nw, onw[::-1])
    bad = rev.copy()
    row0 = set(g.row(0).tolist())
    non = next(x for x in range(1, g.n) if x not in row0)
    bad[uv.shape[0] - 7] = (0, non)
    bad[uv.shape[0] // 3] = (0, non)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan(graph, bad, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    assert ei.value.code == bq.ENOEDGE and f"query {uv.shape[0] // 3}:" in str(ei.value)
    graph.close()


def test_powerlaw_full_size_sampled(env):
    """Chung-Lu n=4M, mean degree 10, exponent 2.1, largest component: all
    edges estimated on the GPU with the scheduled plan at eps=0.05, in the
    launch configuration the bench times; 300 sampled edges bit-exact
    against the oracle (a result depends only on its own edge)."""
    bq, torch = env
    from workloads import cached, chung_lu
    g = cached("chunglu4m_d10_g2.1_s3", lambda: chung_lu(4_000_000, 10, 2.1, seed=3))
    graph = bq.Graph.from_csr(g)
    sched = bq.Schedule(SCHEDULE[0], SCHEDULE[1], SCHEDULE[2], SCHEDULE[3], SCHEDULE[4], 0)
    tau, nw = bq.aesc_plan(graph, None, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    counts, sc = bq.aesc_estimate(graph, 5, None, torch.from_numpy(tau.view(np.int32)).cuda(),
                                  torch.from_numpy(nw.view(np.int32)).cuda())
    bq.sync()
    counts = counts.cpu().numpy().view(np.uint32).reshape(-1, 4)
    sc = sc.cpu().numpy()
    assert np.isfinite(sc).all()
    rng = np.random.default_rng(11)
    pick = np.sort(rng.choice(tau.size, 300, replace=False))
    uv = all_edges(g)[pick]
    ocounts, osc = oracle.aesc_estimate(g, 5, uv, tau[pick], nw[pick])
    assert np.array_equal(counts[pick].ravel(), ocounts)
    assert same_bits(sc[pick], osc)
    graph.close()


def test_errors_nan_and_status(env):
    bq, torch = env
    g = cycle(10)
    graph = bq.Graph.from_csr(g)
    uv = np.array([[0, 1], [0, 5], [3, 4], [7, 7], [2, 99]], np.uint32)
    tau = np.array([4, 4, 0, 4, 4], np.uint32)
    nw = np.array([100, 100, 100, 100, 100], np.uint32)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_host(graph, 1, uv, tau, nw)
    assert ei.value.code in (bq.ENOEDGE, bq.EINVAL)
    # device variant: valid rows finite and equal to the oracle, others NaN
    counts, sc = bq.aesc_estimate(graph, 1, torch.from_numpy(uv.view(np.int32)).cuda(),
                                  torch.from_numpy(tau.view(np.int32)).cuda(),
                                  torch.from_numpy(nw.view(np.int32)).cuda())
    with pytest.raises(bq.BouquetError):
        bq.sync()
    sc = sc.cpu().numpy()
    assert np.isnan(sc[1:]).all()
    _, osc = oracle.aesc_estimate(g, 1, uv[:1], tau[:1], nw[:1])
    assert same_bits(sc[:1], osc)
    big = np.array([1 << 30], np.uint32)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_host(graph, 1, uv[:1], np.array([4], np.uint32), big)
    assert ei.value.code == bq.EOVERFLOW
    bq.sync()


def test_planner_errors(env):
    bq, _ = env
    g = cycle(10)
    graph = bq.Graph.from_csr(g)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan(graph, np.array([[0, 1]], np.uint32), 0.1)
    assert ei.value.code == bq.EINVAL and "spectrum" in str(ei.value)
    _, l2, lneg = exact.spectrum(g)
    graph.set_spectrum(l2, lneg)
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan(graph, np.array([[0, 5]], np.uint32), 0.1)
    assert ei.value.code == bq.ENOEDGE
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_plan(graph, np.array([[0, 1]], np.uint32), 1e-3)
    assert ei.value.code == bq.EOVERFLOW


@pytest.mark.parametrize("omega", [1, 3, 8])
def test_certified_plan_with_eigenvectors(env, omega):
    """bq_graph_set_eigvecs: the library's certified plan equals the oracle's
    omega plan (never longer than the plain plan), and the estimate with it
    meets eps against the exact SC."""
    bq, torch = env
    from oracle import exact
    from workloads import cycle, grid_deleted
    for g in (gnp_connected(14, 0.3, 4), cycle(10), grid_deleted(5, 6, 0.0, 1)):
        graph = bq.Graph.from_csr(g)
        uv = all_edges(g)
        _, l2, lneg = exact.spectrum(g)
        graph.set_spectrum(l2, lneg)
        w = min(omega, g.n - 2)
        lam, vecs, rest, _ = exact.eigen_embedding(g, w)
        graph.set_eigvecs(lam, vecs, rest)
        tau, nw = bq.aesc_plan(graph, uv, 0.1, 0.01)
        otau, onw = oracle.plan_certified_omega(g, uv, 0.1, 0.01, lam, vecs, rest, lneg)
        assert np.array_equal(tau, otau) and np.array_equal(nw, onw)
        graph.set_eigvecs(np.zeros(0), np.zeros(0), 0.0)  # cleared: the plain plan
        ptau, pnw = bq.aesc_plan(graph, uv, 0.1, 0.01)
        assert np.all(tau <= ptau) and np.all(nw <= pnw)
        counts, sc = bq.aesc_estimate_host(graph, 31, uv, tau, nw)
        assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= 0.1
        with pytest.raises(bq.BouquetError):
            graph.set_eigvecs(np.array([1.0]), np.zeros(g.n), 0.0)  # eigenvalue 1 is excluded
        graph.close()
