"""Pins of the certified plan with omega known eigenpairs (CalculateTau's
eigenvector refinement): with every eigenpair the bound is the exact
truncation error of the half-weighted series; with none it is the plain
plan; in between it certifies (error at the planned tau within eps / 2) with
a tau no longer than the plain plan's."""

import numpy as np
import pytest

import oracle
from oracle import exact
from workloads import all_edges, complete, cycle, diamond, gnp_connected, grid_deleted, prufer_tree

def plan_or_code(f):
    """The plan, or the oracle's error code (EOVERFLOW when 2 N tau >= 2^32)."""
    try:
        return f()
    except oracle.OracleError as e:
        return e.code


GRAPHS = [complete(8), cycle(10), diamond(), prufer_tree(12, 2), gnp_connected(14, 0.3, 4),
          grid_deleted(5, 6, 0.0, 1)]


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_full_spectrum_bound_is_the_exact_error(g):
    lam, vecs, rest, lneg = exact.eigen_embedding(g, g.n - 1)
    d = g.degrees
    for u, v in all_edges(g).tolist()[:8]:
        s_e = 1.0 / d[u] + 1.0 / d[v]
        sc = exact.sc_pinv(g, np.array([[u, v]]))[0]
        for tau in (1, 2, 3, 5, 8, 13):
            err = sc - exact.truncated_series(g, u, v, tau)
            b = oracle.trunc_bound_omega(s_e, lam, vecs[u], vecs[v], rest, lneg, tau)
            assert abs(b - abs(err)) < 1e-10, (u, v, tau)


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_omega_zero_is_the_plain_plan(g):
    uv = all_edges(g)
    _, l2, lneg = exact.spectrum(g)
    want = plan_or_code(lambda: oracle.plan_certified(g, uv, 0.1, 0.01, l2, lneg))
    got = plan_or_code(lambda: oracle.plan_certified_omega(g, uv, 0.1, 0.01, np.zeros(0), np.zeros((g.n, 0)),
                                                           l2, lneg))
    if isinstance(want, int):  # the 12-vertex tree overflows 2 N tau < 2^32 at eps = 0.1
        assert got == want
    else:
        assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
@pytest.mark.parametrize("omega", [1, 3])
@pytest.mark.parametrize("eps", [0.1, 0.02])
def test_partial_spectrum_certifies_with_shorter_tau(g, omega, eps):
    uv = all_edges(g)
    _, l2, lneg = exact.spectrum(g)
    omega = min(omega, g.n - 2)
    lam, vecs, rest, lneg2 = exact.eigen_embedding(g, omega)
    assert lneg2 == lneg
    plain = plan_or_code(lambda: oracle.plan_certified(g, uv, eps, 0.01, l2, lneg))
    got = plan_or_code(lambda: oracle.plan_certified_omega(g, uv, eps, 0.01, lam, vecs, rest, lneg))
    if isinstance(got, int):
        assert isinstance(plain, int)  # overflow with the eigenvectors implies overflow without
        return
    tau, nw = got
    if not isinstance(plain, int):
        assert np.all(tau <= plain[0]) and np.all(nw <= plain[1])
    sc = exact.sc_pinv(g, uv)
    for (u, v), t, want in zip(uv.tolist(), tau, sc):
        assert abs(want - exact.truncated_series(g, u, v, int(t))) <= eps / 2 + 1e-12
