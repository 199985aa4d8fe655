"""Pins of the oracle's exact references (spanning-tree counts, effective
resistance, spectrum, truncated walk series) against closed forms, textbook
counts and the worked example of Fig. 1."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact
from tests.conftest import golden_rows
from workloads import (all_edges, complete, cycle, diamond, edges_of, er_with_path,
                       gnp_connected, grid_deleted, path, prufer_tree)


def edge_list(g):
    u, v = edges_of(g)
    return list(zip(u.tolist(), v.tolist()))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_cayley_formula(n):
    # Cayley: K_n has n^(n-2) spanning trees.
    assert exact.spanning_tree_count(n, edge_list(complete(n))) == n ** (n - 2)


@pytest.mark.parametrize("n", [3, 5, 10])
def test_cycle_and_tree_counts(n):
    assert exact.spanning_tree_count(n, edge_list(cycle(n))) == n
    assert exact.spanning_tree_count(n, edge_list(prufer_tree(n, n))) == 1


def test_fig1_diamond_golden():
    rows = golden_rows("fig1_diamond.txt")
    g = diamond()
    want = {(int(r[0]), int(r[1])): Fraction(r[2]) for r in rows if r[0] != "T"}
    total = [int(r[1]) for r in rows if r[0] == "T"][0]
    assert exact.spanning_tree_count(4, edge_list(g)) == total
    uv = np.array(list(want.keys()), np.uint32)
    got = exact.sc_matrix_tree(g, uv)
    assert dict(zip(want.keys(), got)) == want
    pinv = exact.sc_pinv(g, uv)
    assert np.allclose(pinv, [float(x) for x in want.values()], atol=1e-12)
    # the caption's "all edges 1/2" contradicts Foster's theorem (sum = n-1)
    assert sum(got) == 3


@pytest.mark.parametrize("g", [prufer_tree(12, 2), gnp_connected(10, 0.5, 3), diamond(),
                               cycle(7), complete(6)], ids=lambda g: g.name)
def test_pinv_equals_matrix_tree(g):
    uv = all_edges(g)
    brute = np.array([float(x) for x in exact.sc_matrix_tree(g, uv)])
    assert np.allclose(exact.sc_pinv(g, uv), brute, atol=1e-12)


def test_closed_forms():
    for n in (4, 8, 13):
        sc = exact.sc_pinv(complete(n), all_edges(complete(n)))
        assert np.allclose(sc, 2.0 / n, atol=1e-12)
        sc = exact.sc_pinv(cycle(n), all_edges(cycle(n)))
        assert np.allclose(sc, (n - 1) / n, atol=1e-12)
    t = prufer_tree(12, 2)
    assert np.allclose(exact.sc_pinv(t, all_edges(t)), 1.0, atol=1e-12)
    # a bridge joining two triangles has SC 1; triangle edges 2/3
    from workloads import csr_from_edges
    g = csr_from_edges(6, [0, 1, 2, 3, 4, 5, 2], [1, 2, 0, 4, 5, 3, 3])
    sc = dict(zip(map(tuple, all_edges(g).tolist()), exact.sc_pinv(g, all_edges(g))))
    assert abs(sc[(2, 3)] - 1.0) < 1e-12
    assert abs(sc[(0, 1)] - 2.0 / 3.0) < 1e-12


def test_foster_on_tiny_aesc_graph():
    g = er_with_path(1000, 5000, 1)
    sc = exact.sc_pinv(g, all_edges(g))
    assert abs(sc.sum() - (g.n - 1)) < 1e-7
    assert np.all(sc > 0) and np.all(sc <= 1 + 1e-12)


def test_spectrum_closed_forms():
    lam, l2, lneg = exact.spectrum(complete(8))
    assert abs(l2 + 1.0 / 7.0) < 1e-12 and abs(lneg + 1.0 / 7.0) < 1e-12
    assert abs(lam[-1] - 1.0) < 1e-12
    lam, l2, lneg = exact.spectrum(cycle(10))
    want = np.sort(np.cos(2 * np.pi * np.arange(10) / 10))
    assert np.allclose(lam, want, atol=1e-12)
    assert abs(l2 - math.cos(math.pi / 5)) < 1e-12
    assert abs(lneg + math.cos(math.pi / 5)) < 1e-12  # -1 removed (bipartite)
    lam, l2, lneg = exact.spectrum(cycle(9))  # odd cycle: no -1 to remove
    assert abs(lneg - math.cos(8 * math.pi / 9)) < 1e-12
    assert exact.is_bipartite(prufer_tree(12, 2)) and not exact.is_bipartite(cycle(9))


@pytest.mark.parametrize("g", [complete(8), cycle(10), cycle(9), diamond(),
                               prufer_tree(12, 2), gnp_connected(10, 0.5, 3)],
                         ids=lambda g: g.name)
def test_truncated_series_converges_to_sc(g):
    # The half-weighted series tends to R_eff, bipartite graphs included.
    uv = all_edges(g)
    sc = exact.sc_pinv(g, uv)
    for (u, v), want in zip(uv.tolist(), sc):
        assert abs(exact.truncated_series(g, u, v, 400) - want) < 1e-9


def test_half_weight_needed_on_bipartite_cycle():
    # C10: plain partial sums oscillate between two values, the half-weighted
    # series converges (0.8981 at tau = 22, exact 0.9).
    g = cycle(10)
    t = exact.series_terms(g, 0, 1, 401)
    plain_even = t[:400].sum()
    plain_odd = t[:401].sum()
    assert abs(plain_even - plain_odd) > 0.1
    assert abs(exact.truncated_series(g, 0, 1, 22) - 0.8981) < 5e-4
    assert abs(exact.truncated_series(g, 0, 1, 400) - 0.9) < 1e-9


def test_series_term_zero_is_s_e():
    g = gnp_connected(10, 0.5, 3)
    d = g.degrees
    for u, v in all_edges(g).tolist():
        assert abs(exact.series_terms(g, u, v, 0)[0] - (1 / d[u] + 1 / d[v])) < 1e-15


def test_walk_distribution_is_row_of_matrix_power():
    g = diamond()
    P = exact.transition(g)
    assert np.allclose(exact.walk_distribution(g, 1, 3), np.linalg.matrix_power(P, 3)[1])


def test_expected_distinct_ratio_brute_force():
    # E(eta), Sec. 5.6, against enumeration of all beta^alpha outcomes.
    import itertools
    for alpha, beta in [(1, 1), (2, 3), (3, 3), (4, 2), (3, 5)]:
        tot = 0
        for draw in itertools.product(range(beta), repeat=alpha):
            tot += len(set(draw))
        brute = tot / beta ** alpha / alpha
        assert abs(exact.expected_distinct_ratio(alpha, beta) - brute) < 1e-12


def test_path_graph_sc_is_one():
    g = path(6)
    assert np.allclose(exact.sc_pinv(g, all_edges(g)), 1.0)


def test_grid_interior_edges_tend_to_one_half():
    """On the infinite square lattice the effective resistance between
    neighbours is 1/2 (each of the 4 unit currents that enter a node splits
    symmetrically).  The central edge of an s x s grid approaches it from above,
    the gap shrinking like 1/s^2; a corner edge stays far from it."""
    gaps = []
    for side in (21, 31, 41):
        g = grid_deleted(side, side, 0.0, 1)
        c = side // 2
        v0 = c * side + c
        sc = exact.sc_pinv(g, np.array([[v0, v0 + 1], [v0, v0 + side], [0, 1]]))
        assert abs(sc[0] - sc[1]) < 1e-12  # horizontal = vertical by symmetry
        gaps.append(sc[0] - 0.5)
        assert sc[2] > 0.6
    assert 0 < gaps[2] < gaps[1] < gaps[0] < 2e-3
    assert gaps[1] / gaps[0] == pytest.approx((21 / 31) ** 2, rel=0.1)
    # the half-weighted walk series of the central edge heads there too
    g = grid_deleted(21, 21, 0.0, 1)
    v0 = 10 * 21 + 10
    t64 = exact.truncated_series(g, v0, v0 + 1, 64)
    t400 = exact.truncated_series(g, v0, v0 + 1, 400)
    assert abs(t400 - 0.5) < abs(t64 - 0.5) < 0.05
