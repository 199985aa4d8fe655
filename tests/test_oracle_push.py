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


# ------------------------------------------------------------ push depths >= 2

def star_of_paths():
    """An irregular graph (degrees 1 to 4) whose walk laws are not symmetric:
    a hub with four arms of lengths 1..4 and a chord."""
    from workloads import csr_from_edges
    u, v = [], []
    nxt = 1
    for length in range(1, 5):
        prev = 0
        for _ in range(length):
            u.append(prev)
            v.append(nxt)
            prev = nxt
            nxt += 1
    u.append(2)
    v.append(4)
    return csr_from_edges(nxt, np.array(u), np.array(v), name="star_of_paths")


@pytest.mark.parametrize("g", [diamond(), complete(6), cycle(7), prufer_tree(9, 4), gnp_connected(12, 0.4, 5),
                               star_of_paths()], ids=lambda g: g.name)
def test_push_vectors_bound_walk_laws(g):
    """r^j_x(y) lies in [Q p_j(y -> x) - j d_max, Q p_j(y -> x)]: each level
    loses less than one unit per neighbour to the floors.  (A recurrence run
    in the other direction, p_j(x -> y), fails on irregular graphs.)"""
    P = exact.transition(g)
    dmax = int(g.degrees.max())
    Pj = np.eye(g.n)
    for j in range(0, 6):
        for x in range(g.n):
            r = oracle.push_vector(g, x, j).astype(np.float64)
            want = Q * Pj[:, x]
            assert np.all(r <= want + 1e-6) and np.all(r >= want - j * dmax - 1e-6), (x, j)
        Pj = Pj @ P
    # depths 0 and 1 are the closed forms
    for x in range(g.n):
        assert np.array_equal(oracle.push_vector(g, x, 0), push_vector(g, x, 0).astype(np.uint64))
        assert np.array_equal(oracle.push_vector(g, x, 1), push_vector(g, x, 1).astype(np.uint64))


def expected_estimate_deep(g, u, v, tau, depth):
    """E[SC estimate] at any push depth: exact walk laws of the tau - depth
    step walks, the oracle's pushed vectors, and X = sum over l <= depth of
    w_l (r^l_u(u) - r^l_u(v))."""
    u, v = min(u, v), max(u, v)
    d = g.degrees.astype(np.float64)
    P = exact.transition(g)
    w = lambda l: 2.0 if l < tau else 1.0
    ru = oracle.push_vector(g, u, depth).astype(np.float64)
    rv = oracle.push_vector(g, v, depth).astype(np.float64)
    xu = sum(w(l) * (float(oracle.push_vector(g, u, l)[u]) - float(oracle.push_vector(g, u, l)[v]))
             for l in range(depth + 1))
    xv = sum(w(l) * (float(oracle.push_vector(g, v, l)[v]) - float(oracle.push_vector(g, v, l)[u]))
             for l in range(depth + 1))
    E = {"uu": 0.0, "uv": 0.0, "vu": 0.0, "vv": 0.0}
    lu, lv = np.eye(g.n)[u], np.eye(g.n)[v]
    for l in range(1, tau - depth + 1):
        lu, lv = lu @ P, lv @ P
        E["uu"] += w(l + depth) * lu @ ru
        E["uv"] += w(l + depth) * lu @ rv
        E["vu"] += w(l + depth) * lv @ ru
        E["vv"] += w(l + depth) * lv @ rv
    return (xu + E["uu"] - E["vu"]) / (2.0 * Q * d[u]) + (xv + E["vv"] - E["uv"]) / (2.0 * Q * d[v])


@pytest.mark.parametrize("g", [diamond(), complete(6), cycle(8), prufer_tree(9, 4), gnp_connected(12, 0.4, 5),
                               star_of_paths()], ids=lambda g: g.name)
@pytest.mark.parametrize("depth", [2, 3, 5])
def test_deep_expectation_is_truncated_series(g, depth):
    """At every depth the estimator's expectation is the half-weighted series
    (up to the floors' loss, below 1e-6 here)."""
    for u, v in all_edges(g).tolist()[:5]:
        for tau in range(depth, depth + 4):
            want = exact.truncated_series(g, u, v, tau)
            assert abs(expected_estimate_deep(g, u, v, tau, depth) - want) < 1e-6, (u, v, tau)


def test_deep_estimate_without_walks_is_exact():
    """tau = depth: no walk is left and the estimate is X alone, equal to the
    expectation computed from the pushed vectors."""
    g = gnp_connected(12, 0.4, 5)
    uv = all_edges(g)
    for t in (2, 3):
        tau = np.full(uv.shape[0], t, np.uint32)
        nw = np.full(uv.shape[0], 60000, np.uint32)  # volume far below 2N: full depth
        depth, acc, sc = oracle.aesc_push_estimate(g, 1, uv, tau, nw, push_max=t)
        assert np.all(depth == t) and not acc.any()
        for (u, v), s in zip(uv.tolist(), sc):
            assert abs(s - expected_estimate_deep(g, u, v, t, t)) < 1e-12
            assert abs(s - exact.truncated_series(g, u, v, t)) < 1e-6


def support_and_volume(g, x, j):
    supp = [np.count_nonzero(oracle.push_vector(g, x, i)) for i in range(j + 1)]
    vol = [0]
    for i in range(1, j + 1):
        r = oracle.push_vector(g, x, i - 1)
        vol.append(vol[-1] + int(g.degrees[r > 0].sum()))
    return supp, vol


def test_depth_rule_general():
    g = er_with_path(80, 300, 2)
    uv = all_edges(g)[:60]
    rng = np.random.default_rng(3)
    tau = rng.integers(1, 8, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(1, 400, uv.shape[0]).astype(np.uint32)
    for push_max in (2, 4, 8):
        depth, _ = oracle.aesc_push_counts(g, 1, uv, tau, nw, push_max=push_max)
        for q, (a, b) in enumerate(uv.tolist()):
            top = min(push_max, int(tau[q]), 8)
            su, vu = support_and_volume(g, a, top)
            sv, vv = support_and_volume(g, b, top)
            want = 0
            for j in range(1, top + 1):
                if vu[j] + vv[j] >= 2 * int(nw[q]):
                    break
                if j >= 2 and max(su[1:j + 1] + sv[1:j + 1]) > oracle.PUSH_SUPPORT_CAP:
                    break
                want = j
            assert depth[q] == want, (q, push_max)
        if push_max >= 4:
            assert np.any(depth >= 2) and np.any(depth <= 1)


def test_deep_monte_carlo_mean_and_spread():
    g = gnp_connected(14, 0.45, 7)
    uv = all_edges(g)[:4]
    tau = np.full(uv.shape[0], 5, np.uint32)
    nw = np.full(uv.shape[0], 400, np.uint32)
    runs = {pm: np.array([oracle.aesc_push_estimate(g, s, uv, tau, nw, push_max=pm)[2] for s in range(40)])
            for pm in (1, 3)}
    dep = oracle.aesc_push_counts(g, 0, uv, tau, nw, push_max=3)[0]
    assert np.all(dep == 3)
    for i, (u, v) in enumerate(uv.tolist()):
        e = expected_estimate_deep(g, u, v, 5, 3)
        x = runs[3][:, i]
        assert abs(x.mean() - e) < 5 * x.std() / np.sqrt(40) + 1e-9
    assert runs[3].std(axis=0).mean() < runs[1].std(axis=0).mean()


@pytest.mark.parametrize("g,eps", [(complete(8), 0.1), (cycle(10), 0.1), (diamond(), 0.1),
                                   (gnp_connected(10, 0.5, 3), 0.1)], ids=lambda x: getattr(x, "name", str(x)))
def test_deep_eps_contract_with_certified_plan(g, eps):
    uv = all_edges(g)
    _, l2, lneg = exact.spectrum(g)
    tau, nw = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
    depth, _, sc = oracle.aesc_push_estimate(g, 11, uv, tau, nw, push_max=8)
    assert np.max(np.abs(sc - exact.sc_pinv(g, uv))) <= eps


def test_push_max_range():
    g = cycle(6)
    uv = all_edges(g)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.aesc_push_counts(g, 1, uv, np.full(6, 3, np.uint32), np.full(6, 9, np.uint32), push_max=9)
    assert ei.value.code == oracle.EINVAL


def test_support_cap_limits_depth():
    """Depths >= 2 need every level's support within the cap: a star with 600
    leaves stops at depth 1 (level 1 holds the 600 leaves); a two-level tree
    with 30 x 30 grandchildren stops at depth 2 only where level 2 fits."""
    from workloads import csr_from_edges
    star = csr_from_edges(601, np.zeros(600, np.int64), np.arange(1, 601), name="star600")
    uv = all_edges(star)[:5]
    big = np.full(uv.shape[0], 100000, np.uint32)
    depth, _ = oracle.aesc_push_counts(star, 1, uv, np.full(uv.shape[0], 4, np.uint32), big, push_max=4)
    assert np.all(depth == 1)
    # root 0 -> 30 children -> 30 grandchildren each
    u, v = [], []
    nxt = 31
    for c in range(1, 31):
        u.append(0)
        v.append(c)
        for _ in range(30):
            u.append(c)
            v.append(nxt)
            nxt += 1
    tree = csr_from_edges(nxt, np.array(u), np.array(v), name="tree30x30")
    assert np.count_nonzero(oracle.push_vector(tree, 0, 2)) > oracle.PUSH_SUPPORT_CAP or \
        np.count_nonzero(oracle.push_vector(tree, 1, 2)) > oracle.PUSH_SUPPORT_CAP
    q = np.array([[0, 1], [1, 31]], np.uint32)
    depth, _ = oracle.aesc_push_counts(tree, 1, q, np.full(2, 4, np.uint32), np.full(2, 100000, np.uint32),
                                       push_max=4)
    for (a, b), dep in zip(q.tolist(), depth.tolist()):
        s = [max(np.count_nonzero(oracle.push_vector(tree, a, j)), np.count_nonzero(oracle.push_vector(tree, b, j)))
             for j in range(5)]
        want = 1
        for j in range(2, 5):
            if max(s[1:j + 1]) > oracle.PUSH_SUPPORT_CAP:
                break
            want = j
        assert dep == want and dep < 4


@pytest.mark.parametrize("cap", [0, 1, 3, 40, 512])
def test_support_cap_is_a_planner_parameter(cap):
    """The cap is a parameter of the depth rule (0: none, TGT+'s volume rule
    alone).  Without it the 600-leaf star goes as deep as the volumes allow;
    every cap gives the depth recomputed from supports and volumes, and the
    estimator keeps its expectation at whatever depth is taken."""
    g = er_with_path(60, 200, 4)
    uv = all_edges(g)[:40]
    rng = np.random.default_rng(cap + 1)
    tau = rng.integers(2, 7, uv.shape[0]).astype(np.uint32)
    nw = rng.integers(50, 3000, uv.shape[0]).astype(np.uint32)
    depth, _ = oracle.aesc_push_counts(g, 1, uv, tau, nw, push_max=8, support_cap=cap)
    for q, (a, b) in enumerate(uv.tolist()):
        top = min(8, int(tau[q]))
        su, vu = support_and_volume(g, a, top)
        sv, vv = support_and_volume(g, b, top)
        want = 0
        for j in range(1, top + 1):
            if vu[j] + vv[j] >= 2 * int(nw[q]):
                break
            if j >= 2 and cap and max(su[1:j + 1] + sv[1:j + 1]) > cap:
                break
            want = j
        assert depth[q] == want, (q, cap)
    if cap in (1, 3):
        assert depth.max() <= 1 or cap == 3
    from workloads import csr_from_edges
    star = csr_from_edges(601, np.zeros(600, np.int64), np.arange(1, 601), name="star600")
    suv = all_edges(star)[:3]
    sd, _ = oracle.aesc_push_counts(star, 1, suv, np.full(3, 4, np.uint32), np.full(3, 100000, np.uint32),
                                    push_max=4, support_cap=cap)
    assert np.all(sd == (4 if cap == 0 else 1)), sd
    # the expectation at the depth taken is still the half-weighted series
    for (u, v), dep, t in list(zip(uv.tolist(), depth.tolist(), tau.tolist()))[:6]:
        if dep >= 2:
            assert abs(expected_estimate_deep(g, u, v, t, dep) - exact.truncated_series(g, u, v, t)) < 1e-6
