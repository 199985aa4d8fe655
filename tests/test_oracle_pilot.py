"""Pins of the oracle's pilot plan (the scheduled plan's walk count from a
pilot sample): the moment sums against the pinned counters and a Python walk
loop, their expectations against exact walk distributions, the variance
formula against numpy's sample statistics, a closed form on K_n and the
estimator's spread over seeds, and the degenerate and invalid cases."""

import numpy as np
import pytest

import oracle
from workloads import all_edges, complete, cycle, diamond, er_with_path, gnp_connected, path


def walk_scores(g, seed, u, v, side, tau, n0):
    """(a, b) of each of the first n0 walks of one side of edge {u, v}, by a
    Python walk loop on the pinned hash primitives (independent sampler)."""
    e = int(oracle.edge_ids(g, np.array([[u, v]], np.uint32))[0])
    stream = 2 * e + side
    a = np.zeros(n0, np.int64)
    b = np.zeros(n0, np.int64)
    for w in range(n0):
        kw = oracle.walk_key(seed, stream, w)
        cur = u if side == 0 else v
        for l in range(1, tau + 1):
            row = g.row(cur)
            cur = int(row[oracle.choose(oracle.step_hash(kw, l, cur), row.size)])
            wt = 2 if l < tau else 1
            a[w] += wt if cur == u else 0
            b[w] += wt if cur == v else 0
    return a, b


def score_law(g, start, u, v, tau):
    """Exact law of (a, b) for a tau-step simple random walk from start:
    {(a, b): probability}, by dynamic programming over (vertex, a, b)."""
    states = {(start, 0, 0): 1.0}
    for l in range(1, tau + 1):
        wt = 2 if l < tau else 1
        nxt = {}
        for (cur, a, b), p in states.items():
            row = g.row(cur)
            for y in row.tolist():
                key = (y, a + (wt if y == u else 0), b + (wt if y == v else 0))
                nxt[key] = nxt.get(key, 0.0) + p / row.size
        states = nxt
    law = {}
    for (_, a, b), p in states.items():
        law[(a, b)] = law.get((a, b), 0.0) + p
    return law


def law_moment(law, f):
    return sum(p * f(a, b) for (a, b), p in law.items())


def exact_sample_variance(g, u, v, tau):
    """Var Y of one sample of the estimator, Y = ((a(U) - a(V))/d_u +
    (b(V) - b(U))/d_v) / 2 with independent walks U from u and V from v."""
    du, dv = g.row(u).size, g.row(v).size
    total = 0.0
    for start in (u, v):
        law = score_law(g, start, u, v, tau)
        m = law_moment(law, lambda a, b: a / du - b / dv)
        m2 = law_moment(law, lambda a, b: (a / du - b / dv) ** 2)
        total += m2 - m * m
    return total / 4.0


@pytest.mark.parametrize("sampler", [None, (1, 8, 32), (1, 32, 4)], ids=["ind", "coupled8", "coupled32"])
def test_moment_sums_are_the_counters(sampler):
    g = er_with_path(60, 150, 3)
    uv = all_edges(g)
    rng = np.random.default_rng(5)
    tau = rng.integers(1, 9, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 100, uv.shape[0]).astype(np.uint32)
    mo = oracle.aesc_moments(g, 9, uv, tau, nw, sampler)
    counts = oracle.aesc_counts(g, 9, uv, tau, nw, sampler).reshape(-1, 2, 2)
    assert np.array_equal(mo[:, :, 0], counts[:, :, 0].astype(np.uint64))
    assert np.array_equal(mo[:, :, 1], counts[:, :, 1].astype(np.uint64))
    # a^2 >= a and b^2 >= b for integer scores; a b <= (a^2 + b^2) / 2
    assert np.all(mo[:, :, 2] >= mo[:, :, 0]) and np.all(mo[:, :, 3] >= mo[:, :, 1])
    assert np.all(2 * mo[:, :, 4] <= mo[:, :, 2] + mo[:, :, 3])


@pytest.mark.parametrize("g", [diamond(), gnp_connected(12, 0.4, 5)], ids=lambda g: g.name)
def test_moments_equal_python_walk_loop(g):
    uv = all_edges(g)[:5]
    tau = np.array([1, 2, 3, 5, 7][:uv.shape[0]], np.uint32)
    n0 = 40
    mo = oracle.aesc_moments(g, 21, uv, tau, np.full(uv.shape[0], n0, np.uint32))
    for q, (u, v) in enumerate(uv.tolist()):
        for side in (0, 1):
            a, b = walk_scores(g, 21, u, v, side, int(tau[q]), n0)
            want = [a.sum(), b.sum(), (a * a).sum(), (b * b).sum(), (a * b).sum()]
            assert mo[q, side].tolist() == [int(x) for x in want], (q, side)


@pytest.mark.parametrize("g", [diamond(), cycle(7), complete(5)], ids=lambda g: g.name)
def test_moments_converge_to_exact_law(g):
    """Sample means of a, b, a^2, b^2, a b over many pilot walks match the
    exact walk law within 5 standard errors."""
    n0 = 20000
    uv = all_edges(g)[:3]
    tau = np.full(uv.shape[0], 4, np.uint32)
    mo = oracle.aesc_moments(g, 4, uv, tau, np.full(uv.shape[0], n0, np.uint32))
    fs = [lambda a, b: a, lambda a, b: b, lambda a, b: a * a, lambda a, b: b * b, lambda a, b: a * b]
    for q, (u, v) in enumerate(uv.tolist()):
        for side, start in enumerate((u, v)):
            law = score_law(g, start, u, v, 4)
            for i, f in enumerate(fs):
                mean = law_moment(law, f)
                var = law_moment(law, lambda a, b: f(a, b) ** 2) - mean * mean
                got = float(mo[q, side, i]) / n0
                assert abs(got - mean) <= 5 * np.sqrt(var / n0) + 1e-12, (q, side, i)


def test_variance_formula_matches_numpy_sample_statistics():
    g = gnp_connected(12, 0.4, 5)
    uv = all_edges(g)[:4]
    tau = np.array([2, 3, 4, 6], np.uint32)
    n0 = 300
    mo = oracle.aesc_moments(g, 8, uv, tau, np.full(uv.shape[0], n0, np.uint32))
    _, var = oracle.pilot_nwalks(g, uv, tau, mo, n0, 0.1, 3.0, 1)
    for q, (u, v) in enumerate(uv.tolist()):
        du, dv = g.row(u).size, g.row(v).size
        total = 0.0
        for side in (0, 1):
            a, b = walk_scores(g, 8, u, v, side, int(tau[q]), n0)
            c = np.cov(np.stack([a, b]).astype(np.float64), ddof=1)
            total += c[0, 0] / du ** 2 + c[1, 1] / dv ** 2 - 2 * c[0, 1] / (du * dv)
        assert var[q] == pytest.approx(total / 4.0, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("n", [5, 8])
def test_complete_graph_closed_form(n):
    """K_n, tau = 1: a walk from u is on v after one step with probability
    p = 1/(n-1) and never on u, so Var Y = 2 p (1 - p) / (4 d^2), d = n - 1;
    N is z^2 Var Y / (eps/2)^2 rounded up."""
    g = complete(n)
    uv = all_edges(g)[:3]
    tau = np.ones(uv.shape[0], np.uint32)
    n0 = 100000
    mo = oracle.aesc_moments(g, 2, uv, tau, np.full(uv.shape[0], n0, np.uint32))
    eps, z = 0.01, 3.0
    nw, var = oracle.pilot_nwalks(g, uv, tau, mo, n0, eps, z, 1)
    p, d = 1.0 / (n - 1), n - 1
    want = 2 * p * (1 - p) / (4 * d * d)
    assert np.allclose(var, want, rtol=0.05)
    assert np.allclose(nw, np.ceil(z * z * var / (eps / 2) ** 2), rtol=0, atol=0)
    assert np.allclose(nw, z * z * want / (eps / 2) ** 2, rtol=0.05)
    assert exact_sample_variance(g, 0, 1, 1) == pytest.approx(want, rel=1e-12)


def test_estimator_spread_over_seeds_is_variance_over_n():
    """The variance the pilot estimates is the one of the estimate: over many
    seeds, Var(SC estimate with N walks) = Var Y / N (chi-square bounds)."""
    g = gnp_connected(10, 0.5, 3)
    uv = all_edges(g)[:3]
    tau = np.full(uv.shape[0], 3, np.uint32)
    N = 64
    nw = np.full(uv.shape[0], N, np.uint32)
    est = np.array([oracle.aesc_estimate(g, s, uv, tau, nw)[1] for s in range(400)])
    for q, (u, v) in enumerate(uv.tolist()):
        ratio = est[:, q].var(ddof=1) / (exact_sample_variance(g, u, v, 3) / N)
        assert 0.7 < ratio < 1.35, (q, ratio)
    mo = oracle.aesc_moments(g, 77, uv, tau, np.full(uv.shape[0], 50000, np.uint32))
    _, var = oracle.pilot_nwalks(g, uv, tau, mo, 50000, 0.1, 3.0, 1)
    for q, (u, v) in enumerate(uv.tolist()):
        assert var[q] == pytest.approx(exact_sample_variance(g, u, v, 3), rel=0.05)


@pytest.mark.parametrize("g", [complete(8), cycle(10), diamond(), gnp_connected(10, 0.5, 3)],
                         ids=lambda g: g.name)
def test_pilot_plan_error_against_truncated_series(g):
    """With z = 3 the estimate lies within eps/2 of its expectation (the
    half-weighted truncated series) for nearly all edges."""
    from oracle import exact
    uv = all_edges(g)
    eps = 0.1
    tau, nw, _, _ = oracle.plan_pilot(g, 13, uv, eps, 2.0, 2, 64, 32, 400)
    assert np.all(nw >= 32)
    _, sc = oracle.aesc_estimate(g, 13, uv, tau, nw)
    want = np.array([exact.truncated_series(g, u, v, int(t)) for (u, v), t in zip(uv.tolist(), tau)])
    err = np.abs(sc - want)
    assert np.mean(err <= eps / 2) >= 0.9
    assert err.max() <= eps


def test_zero_variance_takes_n_min():
    """On a single edge every walk alternates between the endpoints, so the
    scores are constant, the variance is 0 and N = n_min."""
    g = path(2)
    uv = all_edges(g)
    tau, nw, mo, var = oracle.plan_pilot(g, 1, uv, 0.05, 2.0, 2, 64, 17, 50)
    assert var[0] == 0.0 and nw[0] == 17
    assert np.all(mo[0, :, 0] * mo[0, :, 0] == 50 * mo[0, :, 2])


def test_invalid_and_overflow():
    g = cycle(10)
    uv = all_edges(g)
    tau = np.full(uv.shape[0], 8, np.uint32)
    mo = oracle.aesc_moments(g, 1, uv, tau, np.full(uv.shape[0], 10, np.uint32))
    for n0, eps, z in ((1, 0.1, 3.0), (10, 0.0, 3.0), (10, 0.1, 0.0)):
        with pytest.raises(oracle.OracleError) as ei:
            oracle.pilot_nwalks(g, uv, tau, mo, n0, eps, z, 1)
        assert ei.value.code == oracle.EINVAL
    with pytest.raises(oracle.OracleError) as ei:
        oracle.pilot_nwalks(g, uv, tau, mo, 10, 1e-6, 3.0, 1)
    assert ei.value.code == oracle.EOVERFLOW
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_moments(g, 1, uv, tau, np.full(uv.shape[0], 1 << 28, np.uint32))
    assert ei.value.code == oracle.EOVERFLOW
