"""Pins of the oracle's walk batch (Alg. 2 / Alg. 3 with counter-keyed
sampling): walk validity, visit-count invariants, purity in (seed, walk id,
start), the exact l-step law P^l, and the distinct-lane statistic E(eta)."""

import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import exact
from workloads import (complete, csr_from_edges, cycle, diamond, gnp_connected, rmat,
                       uniform_starts)


def adjacency_sets(g):
    return [set(g.row(v).tolist()) for v in range(g.n)]


def test_paths_are_walks_and_visits_match():
    g = gnp_connected(40, 0.15, 11)
    starts = uniform_starts(g, 3000, 1)
    vis, paths = oracle.walk_batch(g, 123, starts, 17, want_paths=True)
    adj = adjacency_sets(g)
    assert np.array_equal(paths[:, 0], starts)
    for row in paths[:200]:
        for a, b in zip(row[:-1], row[1:]):
            assert int(b) in adj[int(a)]
    assert vis.sum() == starts.size * 17
    assert np.array_equal(vis, np.bincount(paths[:, 1:].ravel(), minlength=g.n))
    vis0 = oracle.walk_batch(g, 123, starts, 17, include_start=True)
    assert np.array_equal(vis0, vis + np.bincount(starts, minlength=g.n))


def test_visits_accumulate():
    g = cycle(12)
    starts = np.arange(12, dtype=np.uint32)
    v1 = oracle.walk_batch(g, 1, starts, 5)
    v2 = oracle.walk_batch(g, 1, starts, 5, visits=v1.copy())
    assert np.array_equal(v2, 2 * v1)


def test_isolated_start_stays():
    g = csr_from_edges(5, [0, 1], [1, 2])  # vertices 3, 4 isolated
    starts = np.array([3, 4, 0], np.uint32)
    vis, paths = oracle.walk_batch(g, 9, starts, 6, want_paths=True)
    assert np.all(paths[0] == 3) and np.all(paths[1] == 4)
    assert vis[3] == 6 and vis[4] == 6


def test_walk_depends_only_on_seed_id_start():
    g = gnp_connected(30, 0.2, 5)
    starts = uniform_starts(g, 500, 2)
    _, full = oracle.walk_batch(g, 77, starts, 9, want_paths=True)
    # the same walks, other walks replaced: the first 100 rows are unchanged
    other = starts.copy()
    other[100:] = (other[100:] + 1) % g.n
    _, part = oracle.walk_batch(g, 77, other, 9, want_paths=True)
    assert np.array_equal(full[:100], part[:100])
    _, reseeded = oracle.walk_batch(g, 78, starts, 9, want_paths=True)
    assert not np.array_equal(full, reseeded)


def test_start_out_of_range_rejected():
    g = cycle(5)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.walk_batch(g, 1, np.array([5], np.uint32), 3)
    assert ei.value.code == oracle.EINVAL


@pytest.mark.parametrize("g,start,steps", [(complete(8), 0, 2), (cycle(10), 0, 5),
                                           (cycle(10), 3, 6), (diamond(), 0, 3),
                                           (gnp_connected(10, 0.5, 3), 4, 4)],
                         ids=lambda x: getattr(x, "name", str(x)))
def test_l_step_law_matches_matrix_power(g, start, steps):
    walks = 60000
    starts = np.full(walks, start, np.uint32)
    _, paths = oracle.walk_batch(g, 2024 + steps, starts, steps, want_paths=True)
    law = exact.walk_distribution(g, start, steps)
    support = law > 1e-12
    obs = np.bincount(paths[:, steps], minlength=g.n)
    assert obs[~support].sum() == 0  # e.g. parity of C10 positions
    p = stats.chisquare(obs[support], walks * law[support]).pvalue
    assert p > 1e-4


@pytest.mark.parametrize("alpha,beta", [(8, 8), (8, 30), (32, 16), (16, 100)])
def test_distinct_lanes_match_expected_ratio(alpha, beta):
    # alpha independent lanes leave a degree-beta vertex together; the
    # number of distinct next vertices follows E(eta) of Sec. 5.6.
    g = csr_from_edges(beta + 1, np.zeros(beta, np.int64), np.arange(1, beta + 1))
    bouquets = 3000
    starts = np.zeros(alpha * bouquets, np.uint32)
    _, paths = oracle.walk_batch(g, 31, starts, 1, want_paths=True)
    nxt = paths[:, 1].reshape(bouquets, alpha)
    distinct = np.array([len(set(r.tolist())) for r in nxt]) / alpha
    want = exact.expected_distinct_ratio(alpha, beta)
    se = distinct.std(ddof=1) / np.sqrt(bouquets)
    assert abs(distinct.mean() - want) < 5 * se + 1e-9


def test_coupled_sampler_marginal_is_exact():
    # Coupled bouquets (shared top t bits) keep each walk an exact random
    # walk: every walk's position law is still P^l.
    g = gnp_connected(10, 0.5, 3)
    walks, steps = 48000, 3
    starts = np.full(walks, 2, np.uint32)
    law = exact.walk_distribution(g, 2, steps)
    for t in (0, 3, 32):
        _, paths = oracle.walk_batch(g, 5, starts, steps, sampler=(1, t, 8),
                                     want_paths=True)
        # one walk per bouquet of 8 keeps the samples independent
        obs = np.bincount(paths[::8, steps], minlength=g.n)
        sup = law > 0
        p = stats.chisquare(obs[sup], obs.sum() * law[sup]).pvalue
        assert p > 1e-4, t


def test_coupled_sampler_coupling_strength():
    g = complete(20)
    starts = np.zeros(32 * 200, np.uint32)
    _, full = oracle.walk_batch(g, 5, starts, 4, sampler=(1, 32, 32), want_paths=True)
    b = full.reshape(200, 32, 5)
    # t = 32: the whole bouquet moves as one walk
    assert np.all(b == b[:, :1, :])
    _, loose = oracle.walk_batch(g, 5, starts, 4, sampler=(1, 2, 32), want_paths=True)
    _, ind = oracle.walk_batch(g, 5, starts, 4, want_paths=True)

    def distinct(p):
        q = p.reshape(200, 32, 5)[:, :, 1]
        return np.mean([len(set(r.tolist())) for r in q])
    assert distinct(loose) < distinct(ind)


def test_rmat_batch_sum_invariant():
    g = rmat(10, 8, seed=3)
    starts = uniform_starts(g, 5000, 4)
    vis = oracle.walk_batch(g, 1, starts, 64)
    assert int(vis.sum()) == 5000 * 64


def test_paths_by_id_replays_batch_walks():
    g = gnp_connected(50, 0.1, 8)
    starts = uniform_starts(g, 400, 3)
    _, paths = oracle.walk_batch(g, 55, starts, 12, want_paths=True)
    ids = np.array([0, 7, 399, 123, 8], np.uint64)
    sub = oracle.walk_paths_by_id(g, 55, ids, starts[ids.astype(np.int64)], 12)
    assert np.array_equal(sub, paths[ids.astype(np.int64)])
    _, cp = oracle.walk_batch(g, 55, starts, 12, sampler=(1, 4, 8), want_paths=True)
    sub = oracle.walk_paths_by_id(g, 55, ids, starts[ids.astype(np.int64)], 12, sampler=(1, 4, 8))
    assert np.array_equal(sub, cp[ids.astype(np.int64)])


def test_literal_saba_word_collapses_walks():
    """The paper's SABA word taken literally (Eq. select-proposed, one seed
    X_W per walk xor a shared hash of (vertex, length)) decides a walk's
    choices by the top bits of X_W alone on a low-degree graph: on C10
    thousands of walks follow a handful of paths, and the l-step law is far
    from P^l, where independent keys give every one of the 2^8 paths."""
    g = cycle(10)
    starts = np.zeros(4096, np.uint32)
    _, lit = oracle.walk_batch(g, 5, starts, 8, sampler=(2, 0, 1), want_paths=True)
    _, ind = oracle.walk_batch(g, 5, starts, 8, want_paths=True)
    assert len({tuple(r) for r in lit.tolist()}) <= 8
    assert len({tuple(r) for r in ind.tolist()}) == 256
    for row in lit:  # still walks on the graph
        for a, b in zip(row[:-1], row[1:]):
            assert b in g.row(int(a))
    law = exact.walk_distribution(g, 0, 8)
    emp = np.bincount(lit[:, 8], minlength=g.n) / lit.shape[0]
    assert np.abs(emp - law).max() > 0.2


def test_literal_saba_word_is_per_walk_and_not_for_aesc():
    g = rmat(8, 8, seed=1)
    starts = np.arange(200, dtype=np.uint32) % g.n
    starts = starts[np.diff(g.offsets)[starts] > 0]
    _, p1 = oracle.walk_batch(g, 9, starts, 6, sampler=(2, 0, 1), want_paths=True)
    ids = np.arange(starts.size, dtype=np.uint64)[::-1].copy()
    p2 = oracle.walk_paths_by_id(g, 9, ids, starts[::-1].copy(), 6, sampler=(2, 0, 1))
    assert np.array_equal(p2[::-1], p1)
    uv = np.array([[int(g.nbrs[0]), 0]], np.uint32) if g.offsets[1] > 0 else None
    if uv is not None:
        with pytest.raises(oracle.OracleError):
            oracle.aesc_counts(g, 1, uv, np.array([3], np.uint32), np.array([4], np.uint32), sampler=(2, 0, 1))


def test_coupled_groups_are_the_independent_samples():
    """Coupled walks of a group move together where the degree is below 2^t,
    so an AESC estimate over N coupled walks varies like one over N / width
    independent walks; with width x N walks the certified plan's eps
    contract holds again (the groups are the independent samples)."""
    from workloads import all_edges, complete, diamond
    g = gnp_connected(12, 0.4, 5)
    uv = all_edges(g)[:3]
    tau = np.full(uv.shape[0], 3, np.uint32)
    nw = np.full(uv.shape[0], 256, np.uint32)
    ind = np.array([oracle.aesc_estimate(g, s, uv, tau, nw)[1] for s in range(200)])
    cpl = np.array([oracle.aesc_estimate(g, s, uv, tau, nw, (1, 8, 32))[1] for s in range(200)])
    ratio = cpl.var(axis=0, ddof=1) / ind.var(axis=0, ddof=1)
    assert np.all(ratio > 16) and np.all(ratio < 64), ratio
    for h, eps in ((complete(8), 0.1), (diamond(), 0.1), (gnp_connected(10, 0.5, 3), 0.1)):
        uv = all_edges(h)
        _, l2, lneg = exact.spectrum(h)
        tau, nw = oracle.plan_certified(h, uv, eps, 0.01, l2, lneg)
        _, sc = oracle.aesc_estimate(h, 7, uv, tau, (nw * 32).astype(np.uint32), (1, 8, 32))
        assert np.max(np.abs(sc - exact.sc_pinv(h, uv))) <= eps
