"""Pins of the oracle's push-phase AESC estimator (Alg. 1 with push depth 0
or 1): its exact expectation is the half-weighted truncated series, depth 0
is the plain counter estimator scaled by Q, the depth rule is TGT+'s volume
test, and estimates meet the eps contract on the exact cases."""

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import all_edges, complete, cycle, diamond, er_with_path, gnp_connected, prufer_tree

Q = oracle.PUSH_Q


def push_vector(g, x, depth):
    """r_x in fixed point: Q [y == x] (depth 0) or floor(Q / d_y) on the
    neighbours of x (depth 1)."""
    r = np.zeros(g.n)
    if depth == 0:
        r[x] = Q
    else:
        d = g.degrees
        for y in g.row(x).tolist():
            r[y] = Q // int(d[y])
    return r


def expected_estimate(g, u, v, tau, depth):
    """E[SC estimate] from exact walk distributions: row u of P^l gives the
    law of a walk from u after l steps."""
    u, v = min(u, v), max(u, v)
    d = g.degrees.astype(np.float64)
    P = exact.transition(g)
    ru, rv = push_vector(g, u, depth), push_vector(g, v, depth)
    w = lambda l: 2.0 if l < tau else 1.0
    E = {"uu": 0.0, "uv": 0.0, "vu": 0.0, "vv": 0.0}
    xu_law = np.eye(g.n)[u]
    xv_law = np.eye(g.n)[v]
    for l in range(1, tau - depth + 1):
        xu_law = xu_law @ P
        xv_law = xv_law @ P
        E["uu"] += w(l + depth) * xu_law @ ru
        E["uv"] += w(l + depth) * xu_law @ rv
        E["vu"] += w(l + depth) * xv_law @ ru
        E["vv"] += w(l + depth) * xv_law @ rv
    xu = xv = 2.0 * Q
    if depth == 1:
        w1 = 2.0 if tau > 1 else 1.0
        xu -= w1 * (Q // int(d[v]))
        xv -= w1 * (Q // int(d[u]))
    gu = (xu + E["uu"] - E["vu"]) / (2.0 * Q * d[u])
    gv = (xv + E["vv"] - E["uv"]) / (2.0 * Q * d[v])
    return gu + gv


@pytest.mark.parametrize("g", [diamond(), complete(6), cycle(7), cycle(8), prufer_tree(9, 4),
                               gnp_connected(12, 0.4, 5)], ids=lambda g: g.name)
@pytest.mark.parametrize("depth", [0, 1])
def test_expectation_is_truncated_series(g, depth):
    # tau from 1 (depth 1: no walk step left, all exact) up to 9
    for u, v in all_edges(g).tolist()[:6]:
        for tau in (1, 2, 3, 9):
            want = exact.truncated_series(g, u, v, tau)
            got = expected_estimate(g, u, v, tau, depth)
            assert abs(got - want) < 1e-7, (u, v, tau)


def test_depth_zero_is_plain_counters_times_q():
    g = er_with_path(60, 150, 3)
    uv = all_edges(g)
    rng = np.random.default_rng(1)
    tau = rng.integers(1, 10, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 400, uv.shape[0]).astype(np.uint32)
    depth, acc = oracle.aesc_push_counts(g, 17, uv, tau, nw, push_max=0)
    counts = oracle.aesc_counts(g, 17, uv, tau, nw)
    assert not depth.any()
    assert np.array_equal(acc, counts.astype(np.uint64) * np.uint64(Q))


def test_depth_rule_is_volume_against_walks():
    g = er_with_path(80, 300, 2)
    uv = all_edges(g)
    d = g.degrees.astype(np.int64)
    tau = np.full(uv.shape[0], 4, np.uint32)
    nw = (np.arange(uv.shape[0]) % 20 + 1).astype(np.uint32)
    depth, _ = oracle.aesc_push_counts(g, 1, uv, tau, nw, push_max=1)
    vol = d[uv[:, 0]] + d[uv[:, 1]]
    assert np.array_equal(depth, (vol < 2 * nw.astype(np.int64)).astype(np.uint32))
    assert depth.any() and not depth.all()


def test_no_walks_when_tau_one_and_depth_one():
    g = complete(5)
    uv = all_edges(g)
    tau = np.ones(uv.shape[0], np.uint32)
    nw = np.full(uv.shape[0], 50, np.uint32)
    depth, acc, sc = oracle.aesc_push_estimate(g, 3, uv, tau, nw)
    assert depth.all() and not acc.any()
    for (u, v), s in zip(uv.tolist(), sc):
        assert abs(s - exact.truncated_series(g, u, v, 1)) < 1e-8


def test_monte_carlo_mean_and_lower_spread():
    """Many seeds: the push estimate's mean matches its expectation, and its
    spread is below the plain estimator's with the same walks budget."""
    g = gnp_connected(14, 0.45, 7)
    uv = all_edges(g)[:4]
    tau = np.full(uv.shape[0], 4, np.uint32)
    nw = np.full(uv.shape[0], 400, np.uint32)
    push, plain = [], []
    for seed in range(40):
        push.append(oracle.aesc_push_estimate(g, seed, uv, tau, nw)[2])
        plain.append(oracle.aesc_estimate(g, seed, uv, tau, nw)[1])
    push, plain = np.array(push), np.array(plain)
    for i, (u, v) in enumerate(uv.tolist()):
        e = expected_estimate(g, u, v, 4, 1)
        assert abs(push[:, i].mean() - e) < 5 * push[:, i].std() / np.sqrt(40) + 1e-9
    assert push.std(axis=0).mean() < plain.std(axis=0).mean()


@pytest.mark.parametrize("g,eps", [(complete(8), 0.1), (cycle(10), 0.1), (diamond(), 0.1),
                                   (gnp_connected(10, 0.5, 3), 0.1)], ids=lambda x: getattr(x, "name", str(x)))
def test_eps_contract_with_certified_plan(g, eps):
    """A push-phase sample is no wider than a plain one (p_1 <= 1), so the
    certified plan still bounds the error."""
    uv = all_edges(g)
    _, l2, lneg = exact.spectrum(g)
    tau, nw = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
    _, _, sc = oracle.aesc_push_estimate(g, 11, uv, tau, nw)
    want = exact.sc_pinv(g, uv)
    assert np.max(np.abs(sc - want)) <= eps
