"""Pins of the oracle's vertex-centric estimator (walks shared by all query
edges at a vertex): its counters against a Python walk loop on the pinned
hash primitives, its walk counts (the maximum over the edges at a vertex),
its expectation against the half-weighted truncated series, its eps contract
under the certified plan, and its error cases."""

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import all_edges, complete, cycle, diamond, er_with_path, gnp_connected, prufer_tree


def shared_counts_py(g, seed, uv, tau, nw, sampler=None):
    """The shared counters by a Python walk loop: per vertex x the maximum
    walk count and length over its query edges, walk w on stream
    VERTEX_STREAM | x; hits weighted per edge by its own tau."""
    k = uv.shape[0]
    vn, vt, at = {}, {}, {}
    for q, (a, b) in enumerate(uv.tolist()):
        for x in (a, b):
            vn[x] = max(vn.get(x, 0), int(nw[q]))
            vt[x] = max(vt.get(x, 0), int(tau[q]))
            at.setdefault(x, []).append(q)
    counts = np.zeros(4 * k, np.int64)
    nused = np.zeros(2 * k, np.int64)
    for x in sorted(vn):
        stream = oracle.VERTEX_STREAM | x
        ret = np.zeros(vt[x] + 1, np.int64)
        for w in range(vn[x]):
            kw = oracle.walk_key(seed, stream, w)
            kg = oracle.walk_key(seed, stream | (1 << 63), w // sampler[2]) if sampler else 0
            cur = x
            for l in range(1, vt[x] + 1):
                row = g.row(cur)
                r = oracle.step_hash(kw, l, cur)
                if sampler:
                    t = sampler[1]
                    r = oracle.step_hash(kg, l, cur) ^ (0 if t >= 32 else r >> t)
                cur = int(row[oracle.choose(r, row.size)])
                if cur == x:
                    ret[l] += 1
                for q in at[x]:
                    u, v = sorted(uv[q].tolist())
                    other = v if x == u else u
                    if cur == other and l <= tau[q]:
                        counts[4 * q + (1 if x == u else 2)] += 2 if l < tau[q] else 1
        for q in at[x]:
            u, v = sorted(uv[q].tolist())
            c = sum((2 if l < tau[q] else 1) * ret[l] for l in range(1, int(tau[q]) + 1))
            counts[4 * q + (0 if x == u else 3)] = c
            nused[2 * q + (0 if x == u else 1)] = vn[x]
    return counts, nused


@pytest.mark.parametrize("sampler", [None, (1, 8, 4)], ids=["ind", "coupled"])
@pytest.mark.parametrize("g", [diamond(), gnp_connected(12, 0.4, 5), prufer_tree(9, 4)], ids=lambda g: g.name)
def test_counts_equal_python_walk_loop(g, sampler):
    uv = all_edges(g)[:7]
    uv[1::2] = uv[1::2, ::-1]
    rng = np.random.default_rng(3)
    tau = rng.integers(1, 7, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 40, uv.shape[0]).astype(np.uint32)
    counts, nused = oracle.aesc_shared_counts(g, 17, uv, tau, nw, sampler)
    want_c, want_n = shared_counts_py(g, 17, uv, tau, nw, sampler)
    assert counts.tolist() == want_c.tolist()
    assert nused.tolist() == want_n.tolist()


def test_walk_counts_are_the_maximum_at_each_vertex():
    g = er_with_path(60, 150, 3)
    uv = all_edges(g)
    rng = np.random.default_rng(5)
    tau = rng.integers(1, 6, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 50, uv.shape[0]).astype(np.uint32)
    _, nused = oracle.aesc_shared_counts(g, 1, uv, tau, nw)
    best = np.zeros(g.n, np.int64)
    for (a, b), n in zip(uv.tolist(), nw.tolist()):
        best[a] = max(best[a], n)
        best[b] = max(best[b], n)
    lo, hi = uv.min(axis=1), uv.max(axis=1)
    assert np.array_equal(nused[0::2], best[lo]) and np.array_equal(nused[1::2], best[hi])
    assert np.all(nused.reshape(-1, 2) >= nw[:, None])
    # a single query walks exactly its own plan
    _, one = oracle.aesc_shared_counts(g, 1, uv[:1], tau[:1], nw[:1])
    assert one.tolist() == [nw[0], nw[0]]


@pytest.mark.parametrize("g", [diamond(), cycle(7), complete(6), gnp_connected(12, 0.4, 5)], ids=lambda g: g.name)
def test_expectation_is_truncated_series(g):
    """E[C_uu / N_u] = sum_l w_l p_l(u, u) and so on, so the mean estimate
    over seeds is the half-weighted series at each edge's own tau, whatever
    the longer walks its endpoints run for other edges."""
    uv = all_edges(g)[:6]
    rng = np.random.default_rng(11)
    tau = rng.integers(1, 7, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(20, 120, uv.shape[0]).astype(np.uint32)
    est = np.array([oracle.aesc_shared_estimate(g, s, uv, tau, nw)[2] for s in range(150)])
    for i, (u, v) in enumerate(uv.tolist()):
        want = exact.truncated_series(g, u, v, int(tau[i]))
        se = est[:, i].std(ddof=1) / np.sqrt(est.shape[0])
        assert abs(est[:, i].mean() - want) <= 5 * se + 1e-12, (i, est[:, i].mean(), want)


@pytest.mark.parametrize("g,eps", [(complete(8), 0.1), (cycle(10), 0.1), (diamond(), 0.1),
                                   (gnp_connected(10, 0.5, 3), 0.1)], ids=lambda x: getattr(x, "name", str(x)))
def test_eps_contract_with_certified_plan(g, eps):
    """Every edge keeps its own tau and gets at least its N walks per side,
    so the certified plan still bounds the error."""
    uv = all_edges(g)
    _, l2, lneg = exact.spectrum(g)
    tau, nw = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
    _, nused, sc = oracle.aesc_shared_estimate(g, 11, uv, tau, nw)
    assert np.all(nused.reshape(-1, 2) >= nw[:, None])
    assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= eps


def test_fewer_walk_steps_than_per_edge_walks():
    g = er_with_path(200, 900, 2)
    uv = all_edges(g)
    tau, nw = oracle.plan_scheduled(g, uv, 0.1, 2.0, 2, 64, 9.0, 32)
    per_edge = float(np.sum(2.0 * tau * nw))
    vn, vt = np.zeros(g.n), np.zeros(g.n)
    for (a, b), t, n in zip(uv.tolist(), tau.tolist(), nw.tolist()):
        for x in (a, b):
            vn[x], vt[x] = max(vn[x], n), max(vt[x], t)
    assert float(np.sum(vn * vt)) < per_edge


def test_errors():
    g = cycle(10)
    uv = all_edges(g)[:3]
    tau = np.full(3, 3, np.uint32)
    nw = np.full(3, 5, np.uint32)
    dup = np.concatenate([uv, uv[1:2, ::-1]])
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_shared_counts(g, 1, dup, np.full(4, 3, np.uint32), np.full(4, 5, np.uint32))
    assert ei.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_shared_counts(g, 1, np.array([[0, 5]], np.uint32), tau[:1], nw[:1])
    assert ei.value.code == oracle.ENOEDGE
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_shared_counts(g, 1, uv, np.array([3, 0, 3], np.uint32), nw)
    assert ei.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_shared_counts(g, 1, uv, np.full(3, 64, np.uint32), np.full(3, 1 << 26, np.uint32))
    assert ei.value.code == oracle.EOVERFLOW
