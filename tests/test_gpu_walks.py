"""Walk-batch parity: the CUDA kernels (bouquet and naive) against the CPU
oracle, bit for bit, through the C ABI.

Sizes span several warps/blocks with ragged tails; the full-size R-MAT case
(scale 20, 2^24 walks of 64 steps) is checked on sampled walks the oracle
replays one by one, plus properties that hold at any size."""

import numpy as np
import pytest

import oracle
from workloads import csr_from_edges, cycle, gnp_connected, path, rmat, rmat20, uniform_starts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def dev_u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


GRAPHS = {
    "gnp60": gnp_connected(60, 0.1, 1),
    "rmat12": rmat(12, 8, seed=2),
    "cycle10": cycle(10),
    "path7": path(7),
    "isolated": csr_from_edges(9, [0, 1, 2, 5], [1, 2, 0, 6]),
}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("n_walks,n_steps", [(1, 5), (31, 1), (33, 7), (5127, 64), (70001, 3)])
def test_visits_bit_exact(env, name, n_walks, n_steps):
    bq, torch = env
    g = GRAPHS[name]
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(n_walks + n_steps)
    starts = rng.integers(0, g.n, n_walks).astype(np.uint32)  # isolated starts included
    want = oracle.walk_batch(g, 1234, starts, n_steps)
    st = dev_u32(torch, starts)
    for mode in (bq.MODE_BOUQUET, bq.MODE_NAIVE):
        vis = bq.walk_batch(graph, 1234, st, n_steps, mode=mode)
        bq.sync()
        assert np.array_equal(host_u32(vis), want), (name, mode)


@pytest.mark.parametrize("sampler", [None, (1, 3, 8), (1, 32, 32), (1, 0, 5), (2, 0, 1)])
def test_paths_and_start_visits_bit_exact(env, sampler):
    bq, torch = env
    g = GRAPHS["rmat12"]
    graph = bq.Graph.from_csr(g)
    starts = uniform_starts(g, 3001, 4)
    want_v, want_p = oracle.walk_batch(g, 77, starts, 20, sampler=sampler, include_start=True,
                                       want_paths=True)
    st = dev_u32(torch, starts)
    for mode in (bq.MODE_BOUQUET, bq.MODE_NAIVE):
        paths = torch.zeros((3001, 21), dtype=torch.int32, device="cuda")
        vis = bq.walk_batch(graph, 77, st, 20, mode=mode, sampler=sampler, visit_start=True,
                            paths=paths)
        bq.sync()
        assert np.array_equal(host_u32(vis), want_v)
        assert np.array_equal(host_u32(paths), want_p)


def test_zero_steps_and_accumulation(env):
    bq, torch = env
    g = GRAPHS["gnp60"]
    graph = bq.Graph.from_csr(g)
    starts = uniform_starts(g, 500, 9)
    st = dev_u32(torch, starts)
    vis = bq.walk_batch(graph, 5, st, 0, visit_start=True)
    bq.sync()
    assert np.array_equal(host_u32(vis), np.bincount(starts, minlength=g.n))
    vis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    for _ in range(3):
        bq.walk_batch(graph, 5, st, 6, visits=vis)
    bq.sync()
    assert np.array_equal(host_u32(vis), 3 * oracle.walk_batch(g, 5, starts, 6))


def test_tuning_never_changes_results(env):
    bq, torch = env
    g = GRAPHS["rmat12"]
    graph = bq.Graph.from_csr(g)
    starts = uniform_starts(g, 40000, 11)
    want = oracle.walk_batch(g, 3, starts, 12)
    st = dev_u32(torch, starts)
    old = bq.get_tuning()
    try:
        for lanes in (1, 2, 4, 8):
            for agg in (0, 1):
                bq.set_tuning(walk_lanes=lanes, aggregate_visits=agg, l2_hints=agg)
                vis = bq.walk_batch(graph, 3, st, 12)
                bq.sync()
                assert np.array_equal(host_u32(vis), want), (lanes, agg)
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("hub_slots", [0, 1024, 5000, 8192, 13312])
@pytest.mark.parametrize("layout", [0, 1, 2, 3, 4, 5])
def test_every_graph_layout_bit_exact(env, layout, hub_slots):
    """Plain or bit-packed neighbour ids with 8- or 16-byte vertex records,
    8- or 16-byte edge records, with or without the shared-memory hub table:
    many ways to read a step, one result."""
    bq, torch = env
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout, hub_slots=hub_slots)
        for name in ("rmat12", "isolated", "cycle10"):
            g = GRAPHS[name]
            graph = bq.Graph.from_csr(g)
            rng = np.random.default_rng(layout)
            starts = rng.integers(0, g.n, 20011).astype(np.uint32)
            st = dev_u32(torch, starts)
            for sampler in (None, (1, 5, 32), (2, 0, 1)):
                want_v, want_p = oracle.walk_batch(g, 41, starts, 17, sampler=sampler,
                                                   include_start=True, want_paths=True)
                for mode in (bq.MODE_BOUQUET, bq.MODE_NAIVE):
                    paths = torch.zeros((starts.size, 18), dtype=torch.int32, device="cuda")
                    vis = bq.walk_batch(graph, 41, st, 17, mode=mode, sampler=sampler,
                                        visit_start=True, paths=paths)
                    bq.sync()
                    assert np.array_equal(host_u32(vis), want_v), (name, sampler, mode)
                    assert np.array_equal(host_u32(paths), want_p), (name, sampler, mode)
            graph.close()
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("hub_cluster", [2, 4, 8])
@pytest.mark.parametrize("layout", [1, 2, 5])
def test_cluster_hub_table_bit_exact(env, layout, hub_cluster):
    """The hub table spread over a thread-block cluster (distributed shared
    memory): same visits and paths as the oracle for every sampler, with the
    start counted, for every lane count."""
    bq, torch = env
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=layout, hub_slots=2048, hub_cluster=hub_cluster)
        for name in ("rmat12", "isolated", "cycle10"):
            g = GRAPHS[name]
            graph = bq.Graph.from_csr(g)
            rng = np.random.default_rng(hub_cluster)
            starts = rng.integers(0, g.n, 30011).astype(np.uint32)
            st = dev_u32(torch, starts)
            for sampler in (None, (1, 5, 32), (2, 0, 1)):
                want_v, want_p = oracle.walk_batch(g, 43, starts, 13, sampler=sampler,
                                                   include_start=True, want_paths=True)
                for lanes in (1, 2, 4):
                    bq.set_tuning(walk_lanes=lanes)
                    paths = torch.zeros((starts.size, 14), dtype=torch.int32, device="cuda")
                    vis = bq.walk_batch(graph, 43, st, 13, sampler=sampler, visit_start=True, paths=paths)
                    bq.sync()
                    assert np.array_equal(host_u32(vis), want_v), (name, sampler, lanes)
                    assert np.array_equal(host_u32(paths), want_p), (name, sampler, lanes)
            graph.close()
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("count_bits", [0, 1, 3])
@pytest.mark.parametrize("hub8_hubs", [0, 700, 2500])
def test_hub8_kernel_bit_exact(env, hub8_hubs, count_bits):
    """The 8-byte-hub kernel on the relabelled copy of an R-MAT scale 14
    graph (hub_slots 1024: 1365 hubs of 12 bytes, 2047 of 8 bytes by
    default; every vertex of degree >= 64 must be a hub): visits and paths
    equal the oracle's for two samplers and every lane count, with the start
    counted, for several hub counts and with the hubs' count field narrowed
    to 1 and 3 bits, so that counts wrap every 2 or 8 visits (each wrap adds
    2^bits to the visits)."""
    bq, torch = env
    old = bq.get_tuning()
    g = rmat(14, 8, seed=7)
    try:
        bq.set_tuning(layout=5, hub_slots=1024, hub_relabel=1)
        graph = bq.Graph.from_csr(g)
        bq.set_tuning(relabel_hub8=1, hub8_hubs=hub8_hubs, hub8_count_bits=count_bits)
        rng = np.random.default_rng(hub8_hubs + count_bits)
        starts = rng.integers(0, g.n, 40009).astype(np.uint32)  # isolated starts included
        st = dev_u32(torch, starts)
        for sampler in (None, (1, 5, 32)):
            want_v, want_p = oracle.walk_batch(g, 51, starts, 11, sampler=sampler, include_start=True,
                                               want_paths=True)
            for lanes in (1, 2, 4):
                bq.set_tuning(walk_lanes=lanes)
                bq.profile_read()
                paths = torch.zeros((starts.size, 12), dtype=torch.int32, device="cuda")
                vis = bq.walk_batch(graph, 51, st, 11, sampler=sampler, visit_start=True, paths=paths)
                bq.sync()
                assert bq.profile_read()["walk_kernels"]["relabel8"] == 1
                assert np.array_equal(host_u32(vis), want_v), (sampler, lanes)
                assert np.array_equal(host_u32(paths), want_p), (sampler, lanes)
        # too few hubs to cover the high-degree vertices: the 12-byte kernel runs
        bq.set_tuning(hub8_hubs=100)
        bq.profile_read()
        vis = bq.walk_batch(graph, 51, st, 11, visit_start=True)
        bq.sync()
        assert bq.profile_read()["walk_kernels"]["relabel"] == 1
        assert np.array_equal(host_u32(vis), oracle.walk_batch(g, 51, starts, 11, include_start=True))
        graph.close()
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("hub_slots", [1024, 8192])
def test_degree_relabelled_copy_bit_exact(env, hub_slots):
    """The walk kernel on the degree-relabelled copy (hubs found by internal
    id): same visits and paths as the oracle for every sampler and lane
    count, with the start counted, on graphs with isolated vertices and on
    graphs whose vertices are all hubs."""
    bq, torch = env
    old = bq.get_tuning()
    try:
        bq.set_tuning(layout=5, hub_slots=hub_slots, hub_relabel=1)
        for name in ("rmat12", "isolated", "cycle10"):
            g = GRAPHS[name]
            graph = bq.Graph.from_csr(g)
            rng = np.random.default_rng(hub_slots)
            starts = rng.integers(0, g.n, 30011).astype(np.uint32)
            st = dev_u32(torch, starts)
            for sampler in (None, (1, 5, 32), (2, 0, 1)):
                want_v, want_p = oracle.walk_batch(g, 47, starts, 13, sampler=sampler,
                                                   include_start=True, want_paths=True)
                for lanes, hub8 in ((1, 0), (2, 0), (4, 0), (1, 1), (2, 1), (4, 1)):
                    bq.set_tuning(walk_lanes=lanes, relabel_hub8=hub8)
                    paths = torch.zeros((starts.size, 14), dtype=torch.int32, device="cuda")
                    vis = bq.walk_batch(graph, 47, st, 13, sampler=sampler, visit_start=True, paths=paths)
                    bq.sync()
                    assert np.array_equal(host_u32(vis), want_v), (name, sampler, lanes, hub8)
                    assert np.array_equal(host_u32(paths), want_p), (name, sampler, lanes, hub8)
                vis = bq.walk_batch(graph, 47, st, 13, sampler=sampler)
                bq.sync()
                assert np.array_equal(host_u32(vis), oracle.walk_batch(g, 47, starts, 13, sampler=sampler))
            graph.close()
    finally:
        bq.set_tuning(**old)


@pytest.mark.parametrize("tuning,kind", [(dict(hub_slots=0, layout=0), "bouquet"),
                                         (dict(hub_slots=1024, layout=5), "hub"),
                                         (dict(hub_slots=1024, layout=5, hub_relabel=1, relabel_hub8=0), "relabel"),
                                         (dict(hub_slots=1024, layout=5, hub_relabel=1, relabel_hub8=1), "relabel8")],
                         ids=["bouquet", "hub", "relabel", "relabel8"])
def test_ungrouped_walks_bit_exact(env, tuning, kind):
    """group_walks = 0: the bouquet kernels run the walks in input order
    (no grouping by start); visits and paths are those of the oracle, and
    starts >= n are skipped and reported as in the grouped path."""
    bq, torch = env
    old = bq.get_tuning()
    g = rmat(12, 8, seed=2)
    try:
        bq.set_tuning(**tuning)
        graph = bq.Graph.from_csr(g)
        bq.set_tuning(group_walks=0)
        rng = np.random.default_rng(17)
        starts = rng.integers(0, g.n, 50021).astype(np.uint32)
        for lanes in (1, 4):
            bq.set_tuning(walk_lanes=lanes)
            want_v, want_p = oracle.walk_batch(g, 61, starts, 12, include_start=True, want_paths=True)
            paths = torch.zeros((starts.size, 13), dtype=torch.int32, device="cuda")
            bq.profile_read()
            vis = bq.walk_batch(graph, 61, dev_u32(torch, starts), 12, visit_start=True, paths=paths)
            bq.sync()
            assert bq.profile_read()["walk_kernels"][kind] == 1
            assert np.array_equal(host_u32(vis), want_v), lanes
            assert np.array_equal(host_u32(paths), want_p), lanes
        bad = starts.copy()
        bad[::997] = g.n + 3
        vis = bq.walk_batch(graph, 61, dev_u32(torch, bad), 12)
        with pytest.raises(bq.BouquetError) as ei:
            bq.sync()
        assert ei.value.code == bq.EINVAL
        keep = bad < g.n
        ids = np.flatnonzero(keep).astype(np.uint64)
        p = oracle.walk_paths_by_id(g, 61, ids, bad[keep], 12)
        want = np.bincount(p[:, 1:].reshape(-1).astype(np.int64), minlength=g.n)
        assert np.array_equal(host_u32(vis).astype(np.int64), want)
        graph.close()
    finally:
        bq.set_tuning(**old)


def test_grouping_with_skewed_starts(env):
    """Grouping by start vertex with skewed starts: thousands of walks on a few
    start vertices beside uniform ones.  The batch equals the oracle, also
    with the literal SABA word, which reorders each start's walks after
    grouping."""
    bq, torch = env
    g = GRAPHS["rmat12"]
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(31)
    starts = np.concatenate([rng.integers(0, 200, 20000), rng.integers(0, g.n, 15000),
                             np.full(9000, 4000)]).astype(np.uint32)
    rng.shuffle(starts)
    st = dev_u32(torch, starts)
    for sampler in (None, (2, 0, 1)):
        want_v, want_p = oracle.walk_batch(g, 19, starts, 9, sampler=sampler, want_paths=True)
        paths = torch.zeros((starts.size, 10), dtype=torch.int32, device="cuda")
        vis = bq.walk_batch(graph, 19, st, 9, sampler=sampler, paths=paths)
        bq.sync()
        assert np.array_equal(host_u32(vis), want_v), sampler
        assert np.array_equal(host_u32(paths), want_p), sampler


def test_host_io_matches_device(env):
    bq, torch = env
    g = GRAPHS["gnp60"]
    graph = bq.Graph.from_csr(g)
    starts = uniform_starts(g, 2000, 12)
    paths = np.zeros((2000, 9), np.uint32)
    vis = bq.walk_batch_host(graph, 8, starts, 8, paths=paths)
    want_v, want_p = oracle.walk_batch(g, 8, starts, 8, want_paths=True)
    assert np.array_equal(vis, want_v) and np.array_equal(paths, want_p)
    base = np.arange(g.n, dtype=np.uint32)
    vis2 = bq.walk_batch_host(graph, 8, starts, 8, visits=base.copy(), mode=bq.MODE_NAIVE)
    assert np.array_equal(vis2, want_v + base)


def test_bad_start_reported_and_skipped(env):
    bq, torch = env
    g = GRAPHS["cycle10"]
    graph = bq.Graph.from_csr(g)
    starts = np.array([0, 3, 10, 5, 99], np.uint32)
    good = starts[starts < g.n]
    for mode in (bq.MODE_BOUQUET, bq.MODE_NAIVE):
        vis = bq.walk_batch(graph, 1, dev_u32(torch, starts), 4, mode=mode)
        with pytest.raises(bq.BouquetError) as ei:
            bq.sync()
        assert ei.value.code == bq.EINVAL
        # each valid walk keeps its own id; the bad ones are skipped
        want = np.zeros(g.n, np.int64)
        for i, s in enumerate(starts):
            if s < g.n:
                p = oracle.walk_paths_by_id(g, 1, np.array([i], np.uint64),
                                            np.array([s], np.uint32), 4)
                want += np.bincount(p[0, 1:], minlength=g.n)
        assert np.array_equal(host_u32(vis), want.astype(np.uint32))
    bq.sync()  # status was cleared
    assert good.size == 3


def test_full_size_rmat_batch(env):
    """R-MAT scale 20 (edge factor 16), 2^24 uniform starts, 64 steps: the
    workload the bench times, in the bench's launch configuration."""
    bq, torch = env
    g = rmat20()
    graph = bq.Graph.from_csr(g)
    n_walks, n_steps = 1 << 24, 64
    starts = uniform_starts(g, n_walks, 21)
    st = dev_u32(torch, starts)
    vb = bq.walk_batch(graph, 2024, st, n_steps, mode=bq.MODE_BOUQUET)
    vn = bq.walk_batch(graph, 2024, st, n_steps, mode=bq.MODE_NAIVE)
    bq.sync()
    assert torch.equal(vb, vn)
    assert int(vb.to(torch.int64).sum()) == n_walks * n_steps
    # paths of every walk: histogram equals the visits; sampled rows equal
    # the oracle's replay of the same walk ids
    paths = torch.empty((n_walks, n_steps + 1), dtype=torch.int32, device="cuda")
    vp = bq.walk_batch(graph, 2024, st, n_steps, mode=bq.MODE_BOUQUET, paths=paths)
    bq.sync()
    assert torch.equal(vp, vb)
    hist = torch.bincount(paths[:, 1:].reshape(-1), minlength=g.n)
    assert torch.equal(hist.to(torch.int32), vb)
    assert torch.equal(paths[:, 0], st)
    rng = np.random.default_rng(5)
    ids = np.sort(rng.choice(n_walks, 3000, replace=False)).astype(np.uint64)
    want = oracle.walk_paths_by_id(g, 2024, ids, starts[ids.astype(np.int64)], n_steps)
    got = host_u32(paths[torch.from_numpy(ids.astype(np.int64)).cuda()])
    assert np.array_equal(got, want)
    del paths
    # the host-buffer path used for the end-to-end number
    vh = bq.walk_batch_host(graph, 2024, starts, n_steps)
    assert np.array_equal(vh, host_u32(vb))


def test_full_size_relabelled_batch_matches_oracle(env):
    """The kernel the bench times, in the bench's configuration: R-MAT scale
    20 (edge factor 16) with its degree-relabelled copy, 2^24 uniform starts,
    64 steps, for 1, 2 and 4 walks per lane.  The copy's 8-byte records pack
    the original id, row offset and degree at the widths this graph needs
    (20, 25 and 9 bits), so this is the size at which those fields are
    exercised.  Visits equal the hashed-hub kernel's and the naive kernel's
    on the plain graph, sum to 2^30, equal the histogram of every path, and
    3000 sampled walks (half starting on a hub of the copy, half not) equal
    the oracle's replay of the same walk ids row for row."""
    bq, torch = env
    g = rmat20()
    n_walks, n_steps = 1 << 24, 64
    starts = uniform_starts(g, n_walks, 21)
    st = dev_u32(torch, starts)
    plain = bq.Graph.from_csr(g)
    vh = bq.walk_batch(plain, 2024, st, n_steps, mode=bq.MODE_BOUQUET)
    vn = bq.walk_batch(plain, 2024, st, n_steps, mode=bq.MODE_NAIVE)
    bq.sync()
    assert torch.equal(vh, vn)
    plain.close()
    old = bq.get_tuning()
    try:
        bq.set_tuning(hub_relabel=1)
        graph = bq.Graph.from_csr(g)
    finally:
        bq.set_tuning(**old)
    info = graph.info()
    assert info["relabel_hubs"] == 10922
    assert (info["relabel_bits_id"], info["relabel_bits_off"], info["relabel_bits_deg"]) == (20, 25, 9)
    deg = np.diff(g.offsets)
    order = np.lexsort((np.arange(g.n), -deg))  # degree descending, then id
    is_hub = np.zeros(g.n, bool)
    is_hub[order[:info["relabel_hubs"]]] = True
    rng = np.random.default_rng(6)
    hub_ids = np.flatnonzero(is_hub[starts])
    other_ids = np.flatnonzero(~is_hub[starts])
    ids = np.sort(np.concatenate([rng.choice(hub_ids, 1500, replace=False),
                                  rng.choice(other_ids, 1500, replace=False)])).astype(np.uint64)
    want = oracle.walk_paths_by_id(g, 2024, ids, starts[ids.astype(np.int64)], n_steps)
    tids = torch.from_numpy(ids.astype(np.int64)).cuda()
    paths = torch.empty((n_walks, n_steps + 1), dtype=torch.int32, device="cuda")
    kernel = {0: "relabel", 1: "relabel8"}
    try:
        for hub8 in (1, 0):
            for lanes in (1, 2, 4):
                bq.set_tuning(walk_lanes=lanes, relabel_hub8=hub8)
                bq.profile_read()
                vr = bq.walk_batch(graph, 2024, st, n_steps, mode=bq.MODE_BOUQUET)
                paths.fill_(-1)
                vp = bq.walk_batch(graph, 2024, st, n_steps, mode=bq.MODE_BOUQUET, paths=paths)
                bq.sync()
                case = (hub8, lanes)
                assert bq.profile_read()["walk_kernels"][kernel[hub8]] == 2, case
                assert torch.equal(vr, vh), case
                assert torch.equal(vp, vh), case
                assert int(vr.to(torch.int64).sum()) == n_walks * n_steps
                hist = torch.bincount(paths[:, 1:].reshape(-1), minlength=g.n)
                assert torch.equal(hist.to(torch.int32), vr), case
                assert torch.equal(paths[:, 0], st), case
                assert np.array_equal(host_u32(paths[tids]), want), case
    finally:
        bq.set_tuning(**old)
        del paths
        graph.close()


def test_literal_saba_word_orders_buckets_and_is_refused_by_aesc(env):
    """The literal SABA sampler: the same paths as the oracle in both modes
    (the bucket ordering by seed changes no result), and AESC calls refuse
    it."""
    bq, torch = env
    from workloads import all_edges
    g = GRAPHS["rmat12"]
    graph = bq.Graph.from_csr(g)
    rng = np.random.default_rng(3)
    live = np.flatnonzero(np.diff(g.offsets) > 0)
    starts = live[rng.integers(0, 40, 30011)].astype(np.uint32)  # big buckets: runs of 1024
    starts[:3000] = live[0]
    want_v, want_p = oracle.walk_batch(g, 12, starts, 9, sampler=(2, 0, 1), want_paths=True)
    st = dev_u32(torch, starts)
    for mode in (bq.MODE_NAIVE, bq.MODE_BOUQUET):
        paths = torch.zeros((starts.size, 10), dtype=torch.int32, device="cuda")
        vis = bq.walk_batch(graph, 12, st, 9, mode=mode, sampler=(2, 0, 1), paths=paths)
        bq.sync()
        assert np.array_equal(host_u32(vis), want_v), mode
        assert np.array_equal(host_u32(paths), want_p), mode
    uv = all_edges(g)[:4]
    with pytest.raises(bq.BouquetError) as ei:
        bq.aesc_estimate_host(graph, 1, uv, np.full(4, 3, np.uint32), np.full(4, 5, np.uint32), sampler=(2, 0, 1))
    assert ei.value.code == bq.EINVAL
