"""The naive one-walk-per-thread AESC kernel (BQ_AESC_NAIVE) against the CPU
oracle and the bouquet kernel, bit for bit, through the C ABI.

Both kernels run the same walks (stream 2 e + side, walk index, sampler);
the naive one gives each walk its own thread on the plain CSR, the bouquet
one advances 32 x lanes walks of one start per warp.  Counters are integers
and the estimates are rounded in the same order, so everything must be
identical: exact cases, the tiny workload, sampled edges of the full
power-law workload, ragged walk counts, the coupled sampler, every layout,
and the error paths."""

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import all_edges, cached, chung_lu, complete, cycle, diamond, er_with_path, gnp_connected, \
    prufer_tree

pytestmark = pytest.mark.gpu


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


def dev_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


EXACT = [("K8", complete(8), 0.1), ("C10", cycle(10), 0.1), ("tree12", prufer_tree(12, 2), 0.2),
         ("gnp10", gnp_connected(10, 0.5, 3), 0.1), ("diamond", diamond(), 0.05)]


@pytest.mark.parametrize("name,g,eps", EXACT, ids=[e[0] for e in EXACT])
def test_naive_exact_cases(env, name, g, eps):
    """Under the certified plan the naive estimate equals the bouquet one and
    lies within eps of the exact SC; with the walk counts capped at 50,000
    (the oracle replays up to 1.35e10 steps otherwise) it equals the
    oracle's counters and estimates."""
    bq, torch = env
    graph = bq.Graph.from_csr(g)
    _, l2, lneg = exact.spectrum(g)
    uv = all_edges(g)
    tau, nw = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
    counts, sc = bq.aesc_estimate_host(graph, 11, uv, tau, nw, naive=True)
    bcounts, bsc = bq.aesc_estimate_host(graph, 11, uv, tau, nw)
    assert np.array_equal(counts, bcounts)
    assert same_bits(sc, bsc)
    assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= eps
    cap = np.minimum(nw, 50_000).astype(np.uint32)
    counts, sc = bq.aesc_estimate_host(graph, 11, uv, tau, cap, naive=True)
    ocounts, osc = oracle.aesc_estimate(g, 11, uv, tau, cap)
    assert np.array_equal(counts, ocounts)
    assert same_bits(sc, osc)
    graph.close()


def test_naive_tiny_workload_equals_bouquet_and_oracle(env):
    """ER n=1000 + spanning path, all 5987 edges, certified eps = 0.1: the
    naive counters equal the bouquet kernel's everywhere and the oracle's on
    300 sampled edges; a reversed subset queried alone gives the same."""
    bq, torch = env
    g = er_with_path(1000, 5000, 1)
    graph = bq.Graph.from_csr(g)
    _, l2, lneg = exact.spectrum(g)
    graph.set_spectrum(l2, lneg)
    uv = all_edges(g)
    tau, nw = bq.aesc_plan(graph, None, 0.1, 0.01)
    t_d, n_d = dev_u32(torch, tau), dev_u32(torch, nw)
    cb, sb = bq.aesc_estimate(graph, 5, None, t_d, n_d)
    cn, sn = bq.aesc_estimate(graph, 5, None, t_d, n_d, naive=True)
    bq.sync()
    assert torch.equal(cb, cn)
    assert same_bits(sb.cpu().numpy(), sn.cpu().numpy())
    rng = np.random.default_rng(1)
    pick = np.sort(rng.choice(uv.shape[0], 300, replace=False))
    ocounts, osc = oracle.aesc_estimate(g, 5, uv[pick], tau[pick], nw[pick])
    assert np.array_equal(cn.cpu().numpy().view(np.uint32).reshape(-1, 4)[pick].ravel(), ocounts)
    assert same_bits(sn.cpu().numpy()[pick], osc)
    c2, s2 = bq.aesc_estimate_host(graph, 5, uv[pick][:, ::-1], tau[pick], nw[pick], naive=True)
    assert np.array_equal(c2, ocounts) and same_bits(s2, osc)
    graph.close()


@pytest.mark.parametrize("sampler", [None, (1, 4, 32), (1, 32, 8), (1, 0, 3)])
def test_naive_ragged_counts_and_samplers(env, sampler):
    """Walk counts from 1 to 700 (not multiples of a warp) and lengths 1..9."""
    bq, torch = env
    g = gnp_connected(30, 0.2, 4)
    graph = bq.Graph.from_csr(g)
    uv = all_edges(g)
    tau = (np.arange(uv.shape[0], dtype=np.uint32) % 9) + 1
    nw = (np.arange(uv.shape[0], dtype=np.uint32) * 37) % 700 + 1
    counts, sc = bq.aesc_estimate_host(graph, 3, uv, tau, nw, sampler=sampler, naive=True)
    ocounts, osc = oracle.aesc_estimate(g, 3, uv, tau, nw, sampler=sampler)
    assert np.array_equal(counts, ocounts) and same_bits(sc, osc)
    graph.close()


@pytest.mark.parametrize("layout", [0, 2, 4, 5])
def test_naive_on_every_layout(env, layout):
    """The naive kernel reads the plain CSR whatever layout the graph has
    (wide records when layout 4 is asked for)."""
    bq, torch = env
    g = gnp_connected(40, 0.15, 6)
    uv = all_edges(g)
    tau = (np.arange(uv.shape[0], dtype=np.uint32) % 9) + 1
    nw = (np.arange(uv.shape[0], dtype=np.uint32) * 53) % 1500 + 1
    want = oracle.aesc_counts(g, 9, uv, tau, nw)
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout)
        graph = bq.Graph.from_csr(g)
        counts, _ = bq.aesc_estimate_host(graph, 9, uv, tau, nw, naive=True)
        assert np.array_equal(counts, want)
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_naive_powerlaw_full_size(env):
    """Chung-Lu n=4M, mean degree 10, exponent 2.1, LCC: all 19.76 M edges
    with the scheduled plan at eps = 0.05, as the bench times it.  The naive
    counters equal the bouquet kernel's for every edge, and 200 sampled
    edges equal the oracle's."""
    bq, torch = env
    g = cached("chunglu4m_d10_g2.1_s3", lambda: chung_lu(4_000_000, 10, 2.1, seed=3))
    graph = bq.Graph.from_csr(g)
    sched = bq.Schedule(2.0, 2, 64, 9.0, 32, 0)
    tau, nw = bq.aesc_plan(graph, None, 0.05, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    t_d, n_d = dev_u32(torch, tau), dev_u32(torch, nw)
    cb, sb = bq.aesc_estimate(graph, 5, None, t_d, n_d)
    cn, sn = bq.aesc_estimate(graph, 5, None, t_d, n_d, naive=True)
    bq.sync()
    assert torch.equal(cb, cn)
    assert torch.equal(sb.view(torch.int64), sn.view(torch.int64))
    rng = np.random.default_rng(12)
    pick = np.sort(rng.choice(tau.size, 200, replace=False))
    uv = all_edges(g)[pick]
    ocounts, osc = oracle.aesc_estimate(g, 5, uv, tau[pick], nw[pick])
    assert np.array_equal(cn.cpu().numpy().view(np.uint32).reshape(-1, 4)[pick].ravel(), ocounts)
    assert same_bits(sn.cpu().numpy()[pick], osc)
    graph.close()


def test_naive_errors_match_bouquet(env):
    """Non-edges, tau = 0 and counters that could wrap give NaN and the same
    status in both kernels; the valid edges are unaffected."""
    bq, torch = env
    g = cycle(10)
    graph = bq.Graph.from_csr(g)
    uv = np.array([[0, 1], [0, 5], [3, 4], [7, 7], [2, 99], [5, 6]], np.uint32)
    tau = np.array([4, 4, 0, 4, 4, 3], np.uint32)
    nw = np.array([100, 100, 100, 100, 100, 77], np.uint32)
    res = []
    for naive in (False, True):
        with pytest.raises(bq.BouquetError) as ei:
            bq.aesc_estimate_host(graph, 2, uv, tau, nw, naive=naive)
        res.append(ei.value.code)
        counts, sc = bq.aesc_estimate(graph, 2, dev_u32(torch, uv), dev_u32(torch, tau), dev_u32(torch, nw),
                                      naive=naive)
        with pytest.raises(bq.BouquetError):
            bq.sync()
        sc = sc.cpu().numpy()
        assert np.isnan(sc[1:5]).all() and np.isfinite(sc[[0, 5]]).all()
        ocounts, osc = oracle.aesc_estimate(g, 2, uv[[0, 5]], tau[[0, 5]], nw[[0, 5]])
        assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(-1, 4)[[0, 5]].ravel(), ocounts)
        assert same_bits(sc[[0, 5]], osc)
    assert res[0] == res[1]
    graph.close()
