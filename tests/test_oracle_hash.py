"""Pins of the oracle's sampler: the hash-keyed neighbour choice of Sec. 3.1 /
Eq. (select-proposed), built from Philox-4x32-10 and the SplitMix64 mixer.

The hashes are pinned to their authors' published known-answer vectors; the
neighbour choice is pinned by its range, by exact equidistribution of the
multiply-high map, and by chi-square tests of uniformity and of step-to-step
independence (the paper used Dieharder for this, Table 2; that suite is not
available here)."""

import numpy as np
import pytest
from scipy import stats

import oracle
from tests.conftest import golden_rows
from workloads import csr_from_edges


def test_philox_known_answers():
    rows = golden_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for row in rows:
        words = [int(x, 16) for x in row]
        ctr, key, want = words[:4], words[4:6], words[6:10]
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_splitmix64_known_answers():
    for row in golden_rows("splitmix64_kat.txt"):
        seed = int(row[0])
        want = [int(x) for x in row[1:]]
        assert oracle.splitmix64_sequence(seed, len(want)) == want


def test_step_hash_is_splitmix_stream_at_vertex_zero():
    # The step word at vertex 0 is the high half of the l-th SplitMix64
    # output for seed = walk key.
    for kw in (0, 1234567, 0xDEADBEEFCAFEBABE):
        seq = oracle.splitmix64_sequence(kw, 6)
        for l in range(1, 7):
            assert oracle.step_hash(kw, l, 0) == seq[l - 1] >> 32


def test_walk_key_is_philox_block_half():
    seed = 0x0123456789ABCDEF
    stream = 0x0000000500000007
    for k in (0, 1, 2, 3, 1001):
        blk = k >> 1
        out = oracle.philox4x32_10(
            [blk & 0xFFFFFFFF, blk >> 32, stream & 0xFFFFFFFF, stream >> 32],
            [seed & 0xFFFFFFFF, seed >> 32])
        lo, hi = (out[2], out[3]) if k & 1 else (out[0], out[1])
        assert oracle.walk_key(seed, stream, k) == int(lo) | (int(hi) << 32)


def test_choose_range_and_boundaries():
    # Eq. (select-proposed) with h_max = 2^32: index k covers exactly the
    # words r with k * 2^32 / d <= r < (k + 1) * 2^32 / d.
    for d in list(range(1, 70)) + [1000, 65535, 1 << 20, (1 << 32) - 1]:
        assert oracle.choose(0, d) == 0
        assert oracle.choose(0xFFFFFFFF, d) == d - 1
        for k in {0, 1, d // 3, d // 2, d - 1}:
            if k == 0 or k >= d:
                continue
            first = -(-(k << 32) // d)  # ceil(k 2^32 / d)
            assert oracle.choose(first, d) == k
            assert oracle.choose(first - 1, d) == k - 1


def test_choose_equidistribution_small_words():
    # With 2^32 replaced by the full word range, each index receives either
    # floor(2^32/d) or ceil(2^32/d) words; check the counts by stepping
    # through the boundaries of every index.
    for d in (3, 5, 7, 10, 12, 33):
        sizes = []
        for k in range(d):
            lo = -(-(k << 32) // d)
            hi = -(-((k + 1) << 32) // d)
            assert oracle.choose(lo, d) == k
            assert oracle.choose(hi - 1, d) == k
            sizes.append(hi - lo)
        assert max(sizes) - min(sizes) <= 1
        assert sum(sizes) == 1 << 32


def star(d):
    return csr_from_edges(d + 1, np.zeros(d, np.int64), np.arange(1, d + 1))


@pytest.mark.parametrize("d", [2, 3, 7, 10, 64])
def test_first_step_uniform_chi2(d):
    g = star(d)
    walks = 4000 * d
    starts = np.zeros(walks, np.uint32)
    _, paths = oracle.walk_batch(g, 99 + d, starts, 1, want_paths=True)
    counts = np.bincount(paths[:, 1].astype(np.int64) - 1, minlength=d)
    assert counts.sum() == walks
    p = stats.chisquare(counts).pvalue
    assert p > 1e-4, (d, counts)


@pytest.mark.parametrize("d", [3, 6])
def test_steps_independent_chi2(d):
    # Star: the walk alternates centre / leaf, so (leaf at step 1, leaf at
    # step 3) is a pair of neighbour choices at the same vertex two steps
    # apart; under the method they are independent and uniform.
    g = star(d)
    walks = 3000 * d * d
    starts = np.zeros(walks, np.uint32)
    _, paths = oracle.walk_batch(g, 7, starts, 3, want_paths=True)
    a = paths[:, 1].astype(np.int64) - 1
    b = paths[:, 3].astype(np.int64) - 1
    table = np.zeros((d, d))
    np.add.at(table, (a, b), 1)
    chi2, p, _, _ = stats.chi2_contingency(table)
    assert p > 1e-4
    p_uniform = stats.chisquare(table.ravel()).pvalue
    assert p_uniform > 1e-4


def test_same_vertex_different_steps_and_walks_differ():
    # The key includes the walk id and the length (Sec. 2.2, Sec. 3.3):
    # a walk returning to the same vertex draws a fresh word.
    kw = oracle.walk_key(5, 11, 0)
    words = {oracle.step_hash(kw, l, 42) for l in range(1, 200)}
    assert len(words) == 199
    keys = {oracle.walk_key(5, 11, k) for k in range(1000)}
    assert len(keys) == 1000
