"""Pins of the oracle's AESC path (Alg. 1 at zero push depth with the
certified plan): hand-derived plans, the truncation bound against the exact
series, the estimator's expectation, and the eps contract against exact SC."""

import math

import numpy as np
import pytest

import oracle
from oracle import exact
from tests.conftest import golden_rows
from workloads import (all_edges, complete, cycle, diamond, er_with_path,
                       gnp_connected, prufer_tree)

GRAPHS = {"K8": complete(8), "C10": cycle(10)}


def plan_for(g, eps, delta=0.01, uv=None):
    uv = all_edges(g) if uv is None else uv
    _, l2, lneg = exact.spectrum(g)
    return uv, oracle.plan_certified(g, uv, eps, delta, l2, lneg)


def test_plan_closed_forms_golden():
    for name, eps, delta, tau, nw in golden_rows("plan_closed_forms.txt"):
        g = GRAPHS[name]
        _, (t, n) = plan_for(g, float(eps), float(delta))
        assert np.all(t == int(tau)), name
        assert np.all(n == int(nw)), name


def test_plan_scheduled_golden():
    for name, eps, ts, ta, tm, ns, nm, tau, nw in golden_rows("plan_scheduled.txt"):
        g = GRAPHS[name]
        t, n = oracle.plan_scheduled(g, all_edges(g), float(eps), float(ts), int(ta), int(tm),
                                     float(ns), int(nm))
        assert np.all(t == int(tau)) and np.all(n == int(nw)), name


def test_plan_scheduled_errors():
    g = cycle(10)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.plan_scheduled(g, np.array([[0, 5]], np.uint32), 0.1, 2.0, 1, 64, 9.0, 1)
    assert ei.value.code == oracle.ENOEDGE
    with pytest.raises(oracle.OracleError) as ei:
        oracle.plan_scheduled(g, np.array([[0, 1]], np.uint32), 1e-4, 2.0, 1, 64, 9.0, 1)
    assert ei.value.code == oracle.EOVERFLOW


@pytest.mark.parametrize("g", [complete(8), cycle(10), cycle(9), diamond(),
                               prufer_tree(12, 2), gnp_connected(10, 0.5, 3)],
                         ids=lambda g: g.name)
def test_truncation_bound_holds_and_tau_minimal(g):
    _, l2, lneg = exact.spectrum(g)
    uv = all_edges(g)
    sc = exact.sc_pinv(g, uv)
    d = g.degrees
    for (u, v), want in zip(uv.tolist(), sc):
        s = 1.0 / d[u] + 1.0 / d[v]
        for tau in range(1, 40):
            err = abs(exact.truncated_series(g, u, v, tau) - want)
            assert err <= oracle.trunc_bound(s, l2, lneg, tau) * (1 + 1e-9) + 1e-14
    checked = 0
    for eps in (0.05, 0.2, 0.5):
        try:
            t, _ = oracle.plan_certified(g, uv, eps, 0.01, l2, lneg)
        except oracle.OracleError as err:  # slow mixing: 2 N tau >= 2^32
            assert err.code == oracle.EOVERFLOW
            continue
        checked += 1
        for (u, v), tq in zip(uv.tolist(), t.tolist()):
            s = 1.0 / d[u] + 1.0 / d[v]
            assert oracle.trunc_bound(s, l2, lneg, tq) <= eps / 2
            if tq > 1:
                assert oracle.trunc_bound(s, l2, lneg, tq - 1) > eps / 2
    assert checked >= 1


def test_negative_side_bound_is_the_maximum():
    # Q(tau) is the maximum of x^tau (1-x) / (2(1+x)) on [0, a]; compare
    # with a dense grid.
    for a in (0.1, 0.5, 0.8, 0.99):
        for tau in (1, 2, 5, 17, 60):
            xs = np.linspace(0, a, 200001)
            grid = np.max(xs ** tau * (1 - xs) / (2 * (1 + xs)))
            q = oracle.trunc_bound(1.0, 0.0, -a, tau)
            assert grid <= q * (1 + 1e-12) and q - grid < 1e-8


def test_plan_errors():
    g = cycle(10)
    _, l2, lneg = exact.spectrum(g)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.plan_certified(g, np.array([[0, 5]], np.uint32), 0.1, 0.01, l2, lneg)
    assert ei.value.code == oracle.ENOEDGE
    with pytest.raises(oracle.OracleError) as ei:  # 2 N tau >= 2^32
        oracle.plan_certified(g, np.array([[0, 1]], np.uint32), 1e-3, 0.01, l2, lneg)
    assert ei.value.code == oracle.EOVERFLOW


def test_edge_ids_canonical():
    g = gnp_connected(10, 0.5, 3)
    uv = all_edges(g)
    assert np.array_equal(oracle.edge_ids(g, uv), np.arange(uv.shape[0]))
    assert np.array_equal(oracle.edge_ids(g, uv[:, ::-1]), np.arange(uv.shape[0]))


@pytest.mark.parametrize("g", [diamond(), prufer_tree(12, 2), gnp_connected(10, 0.5, 3),
                               cycle(9)], ids=lambda g: g.name)
def test_estimator_expectation_is_truncated_series(g):
    # s_e + E[Y] = S_tau: with many samples the estimate sits within a few
    # standard errors (|Y| <= (tau - 1/2) s_e) of the exact series.
    uv = all_edges(g)
    d = g.degrees
    tau = np.full(uv.shape[0], 6, np.uint32)
    nw = np.full(uv.shape[0], 40000, np.uint32)
    counts, est = oracle.aesc_estimate(g, 4242, uv, tau, nw)
    for (u, v), e in zip(uv.tolist(), est):
        s = 1.0 / d[u] + 1.0 / d[v]
        sd = 5.5 * s / math.sqrt(40000)  # (tau - 1/2) s_e bound on |Y|
        assert abs(e - exact.truncated_series(g, u, v, 6)) < 5 * sd


def test_counter_invariants():
    g = gnp_connected(10, 0.5, 3)
    uv = all_edges(g)
    tau = np.full(uv.shape[0], 5, np.uint32)
    nw = np.full(uv.shape[0], 1000, np.uint32)
    c = oracle.aesc_counts(g, 1, uv, tau, nw).reshape(-1, 4)
    # side 0 can stand on u or on v at most once per step
    assert np.all(c[:, 0] + c[:, 1] <= 2 * 1000 * 5)
    assert np.all(c[:, 2] + c[:, 3] <= 2 * 1000 * 5)
    # after an odd number of steps a walk from u ... weights are 2 or 1
    assert np.all(c % 1 == 0)


def test_subset_and_orientation_independent():
    g = gnp_connected(10, 0.5, 3)
    uv = all_edges(g)
    tau = np.full(uv.shape[0], 4, np.uint32)
    nw = np.full(uv.shape[0], 500, np.uint32)
    full = oracle.aesc_counts(g, 9, uv, tau, nw).reshape(-1, 4)
    pick = [5, 1, 7]
    sub = oracle.aesc_counts(g, 9, uv[pick][:, ::-1], tau[pick], nw[pick]).reshape(-1, 4)
    assert np.array_equal(sub, full[pick])


@pytest.mark.parametrize("name,g,eps", [("K8", complete(8), 0.1), ("C10", cycle(10), 0.2),
                                        ("tree12", prufer_tree(12, 2), 0.5),
                                        ("gnp10", gnp_connected(10, 0.5, 3), 0.1),
                                        ("diamond", diamond(), 0.1)])
def test_eps_contract_on_exact_cases(name, g, eps):
    uv, (tau, nw) = plan_for(g, eps)
    _, est = oracle.aesc_estimate(g, 20241018, uv, tau, nw)
    sc = exact.sc_pinv(g, uv)
    assert np.max(np.abs(est - sc)) <= eps, name


@pytest.mark.slow
def test_eps_contract_tiny_aesc_sample():
    # The tiny AESC workload (ER n=1000, m=5000 plus a spanning path) at
    # eps = 0.1 on a sample of 60 edges; spectrum from the exact eigensolver.
    g = er_with_path(1000, 5000, 1)
    uv_all = all_edges(g)
    rng = np.random.default_rng(0)
    uv = uv_all[rng.choice(uv_all.shape[0], 60, replace=False)]
    uv, (tau, nw) = plan_for(g, 0.1, uv=uv)
    _, est = oracle.aesc_estimate(g, 7, uv, tau, nw)
    assert np.max(np.abs(est - exact.sc_pinv(g, uv))) <= 0.1


def test_finalize_rounding_order():
    # s_e + ((C_uu - C_vu)/d_u + (C_vv - C_uv)/d_v) / (2N), each op rounded
    g = diamond()
    uv = np.array([[0, 1]], np.uint32)
    counts = np.array([7, 3, 2, 11], np.uint32)
    got = oracle.aesc_finalize(g, uv, np.array([3], np.uint32), counts)[0]
    du, dv = 2.0, 3.0
    assert got == (1 / du + 1 / dv) + ((7 - 2) / du + (11 - 3) / dv) / 6.0
