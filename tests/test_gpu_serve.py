"""Serving loop: requests on resident graphs with continuous batching.

A request's counters and estimates must be bit-identical to the oracle's
with the scheduled plan and the same seed, whether it runs alone, in a mix
of requests or spread over many small iterations; admission, queue limits,
timeouts and bad requests give the documented statuses."""

import time

import numpy as np
import pytest

import oracle
from workloads import all_edges, gnp_connected, grid_deleted, rmat

pytestmark = pytest.mark.gpu

SCHED = dict(tau_scale=2.0, tau_add=2, tau_max=64, n_scale=9.0, n_min=32)


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    hosts = [gnp_connected(200, 0.05, 9), rmat(12, 8, seed=2), grid_deleted(30, 30, 0.1, 3)]
    graphs = [bq.Graph.from_csr(g) for g in hosts]
    return bq, hosts, graphs


def same_bits(a, b):
    return np.array_equal(np.asarray(a, np.float64).view(np.uint64), np.asarray(b, np.float64).view(np.uint64))


def requests(hosts, rng, count):
    out = []
    for i in range(count):
        gi = i % len(hosts)
        uv_all = all_edges(hosts[gi])
        k = int(rng.integers(1, min(200, uv_all.shape[0]) + 1))
        uv = uv_all[rng.choice(uv_all.shape[0], k, replace=False)]
        if i % 2:
            uv = uv[:, ::-1].copy()
        eps = float(rng.uniform(0.1, 0.3))
        seed = int(rng.integers(0, 2**63))
        out.append((gi, uv, eps, seed))
    return out


def check_against_oracle(hosts, req, sc, counts):
    gi, uv, eps, seed = req
    tau, nw = oracle.plan_scheduled(hosts[gi], uv, eps, **SCHED)
    oc, osc = oracle.aesc_estimate(hosts[gi], seed, uv, tau, nw)
    assert np.array_equal(counts.reshape(-1), oc)
    assert same_bits(sc, osc)


def test_mix_matches_oracle(env):
    bq, hosts, graphs = env
    rng = np.random.default_rng(11)
    reqs = requests(hosts, rng, 18)
    with bq.Server(graphs, tasks_per_iteration=64, **SCHED) as srv:
        ids = [srv.submit(gi, uv, eps, seed) for gi, uv, eps, seed in reqs]
        results = [srv.wait(rid, timeout=120, counts=True) for rid in ids]
        st = srv.stats()
    for req, (sc, counts, lat) in zip(reqs, results):
        assert lat >= 0.0
        check_against_oracle(hosts, req, sc, counts)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["edges_completed"] == sum(r[1].shape[0] for r in reqs)
    assert st["iterations"] > 1 and 0.0 <= st["p50_ms"] <= st["p99_ms"]


def test_alone_equals_mixed_and_single_call(env):
    """The same request alone, in a mix and through bq_aesc_estimate."""
    import torch
    bq, hosts, graphs = env
    rng = np.random.default_rng(5)
    reqs = requests(hosts, rng, 7)
    target = reqs[4]
    with bq.Server(graphs, tasks_per_iteration=3, **SCHED) as srv:
        sc_alone, c_alone, _ = srv.wait(srv.submit(*target), timeout=120, counts=True)
    with bq.Server(graphs, **SCHED) as srv:
        ids = [srv.submit(*r) for r in reqs]
        mixed = [srv.wait(rid, timeout=120, counts=True) for rid in ids]
    sc_mix, c_mix, _ = mixed[4]
    assert np.array_equal(c_alone, c_mix) and same_bits(sc_alone, sc_mix)
    gi, uv, eps, seed = target
    tau, nw = bq.aesc_plan(graphs[gi], uv, eps, mode=bq.PLAN_SCHEDULED, schedule=bq.Schedule(**SCHED))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()
    counts, sc = bq.aesc_estimate(graphs[gi], seed, dev(uv), dev(tau), dev(nw))
    bq.sync()
    assert np.array_equal(counts.cpu().numpy().view(np.uint32).reshape(-1), c_alone.reshape(-1))
    assert same_bits(sc.cpu().numpy(), sc_alone)


def test_pinned_fallbacks_counted(env):
    """Request images that find the page-locked arena full are page-locked on
    demand and counted in the stats, with unchanged results; with the default
    arena and results read as they come, small requests need none."""
    bq, hosts, graphs = env
    rng = np.random.default_rng(21)
    reqs = requests(hosts, rng, 12)
    with bq.Server(graphs, pinned_arena_bytes=4096, **SCHED) as srv:
        ids = [srv.submit(*r) for r in reqs]
        results = [srv.wait(rid, timeout=120, counts=True) for rid in ids]
        st = srv.stats()
    assert st["pinned_fallbacks"] >= 1 and st["pinned_fallback_s"] >= 0.0
    for req, (sc, counts, _) in zip(reqs, results):
        check_against_oracle(hosts, req, sc, counts)
    with bq.Server(graphs, **SCHED) as srv:
        for r in reqs:
            srv.wait(srv.submit(*r), timeout=120)
        assert srv.stats()["pinned_fallbacks"] == 0


def test_empty_and_failed_requests(env):
    bq, hosts, graphs = env
    uv_ok = all_edges(hosts[0])[:5]
    with bq.Server(graphs, **SCHED) as srv:
        empty = srv.submit(0, np.zeros((0, 2), np.uint32), 0.1, 1)
        g0 = hosts[0]
        row0 = set(g0.nbrs[g0.offsets[0]:g0.offsets[1]].tolist())
        non_nbr = next(x for x in range(1, g0.n) if x not in row0)
        for bad in ([[0, 0]], [[0, 1], [g0.n, 1]]):
            with pytest.raises(bq.BouquetError) as ei:
                srv.submit(0, np.array(bad, np.uint32), 0.1, 1)
            assert ei.value.code == bq.ENOEDGE
        # a pair of vertices with neighbours that is not an edge: found on the GPU
        not_edge = srv.submit(0, np.array([uv_ok[0].tolist(), [0, non_nbr]], np.uint32), 0.1, 1)
        ok = srv.submit(0, uv_ok, 0.2, 3)
        sc, _, _ = srv.wait(empty, timeout=60)
        assert sc.size == 0
        with pytest.raises(bq.BouquetError) as ei:
            srv.wait(not_edge, timeout=60)
        assert ei.value.code == bq.ENOEDGE
        sc, counts, _ = srv.wait(ok, timeout=60, counts=True)
        check_against_oracle(hosts, (0, uv_ok, 0.2, 3), sc, counts)
        with pytest.raises(bq.BouquetError) as ei:
            srv.wait(ok, timeout=0)  # each request is returned once
        assert ei.value.code == bq.EINVAL
        st = srv.stats()
        assert st["completed"] == 2 and st["failed"] == 1 and st["submitted"] == 3
        for args in [(7, uv_ok, 0.1, 0), (0, uv_ok, 0.0, 0), (0, uv_ok, float("nan"), 0)]:
            with pytest.raises(bq.BouquetError) as ei:
                srv.submit(*args)
            assert ei.value.code == bq.EINVAL


def test_budget_queue_and_timeout(env):
    bq, hosts, graphs = env
    uv_big = all_edges(hosts[1])
    # a request larger than the whole budget fails with ENOMEM, the rest run
    with bq.Server(graphs, device_budget_bytes=64 << 10, **SCHED) as srv:
        big = srv.submit(1, uv_big, 0.1, 1)
        small = srv.submit(0, all_edges(hosts[0])[:10], 0.2, 2)
        with pytest.raises(bq.BouquetError) as ei:
            srv.wait(big, timeout=60)
        assert ei.value.code == bq.ENOMEM
        sc, counts, _ = srv.wait(small, timeout=60, counts=True)
        check_against_oracle(hosts, (0, all_edges(hosts[0])[:10], 0.2, 2), sc, counts)
    # one request on the GPU at a time and a one-slot queue: a burst of
    # submissions behind a large request meets a full queue
    with bq.Server(graphs, max_inflight=1, max_pending=1, **SCHED) as srv:
        first = srv.submit(1, uv_big, 0.05, 1)
        with pytest.raises(bq.BouquetError) as ei:
            srv.wait(first, timeout=0)
        assert ei.value.code == bq.ETIMEOUT
        accepted, busy = [first], 0
        for i in range(6):
            try:
                accepted.append(srv.submit(0, all_edges(hosts[0])[:4], 0.3, 10 + i))
            except bq.BouquetError as e:
                assert e.code == bq.EBUSY
                busy += 1
        assert busy >= 1
        for rid in accepted:
            srv.wait(rid, timeout=120)
        st = srv.stats()
        assert st["completed"] == len(accepted) and st["pending"] == 0 and st["inflight"] == 0


def test_destroy_finishes_queued_requests(env):
    bq, hosts, graphs = env
    rng = np.random.default_rng(2)
    srv = bq.Server(graphs, **SCHED)
    for req in requests(hosts, rng, 6):
        srv.submit(*req)
    t0 = time.time()
    srv.close()  # joins the worker after the queue drains
    assert time.time() - t0 < 120


def test_concurrent_clients(env):
    """Four client threads submit and wait at once (the binding releases the
    GIL in the library calls); every result equals the oracle's."""
    import concurrent.futures as cf
    bq, hosts, graphs = env
    rng = np.random.default_rng(21)
    reqs = requests(hosts, rng, 24)
    with bq.Server(graphs, tasks_per_iteration=128, planner_threads=3, **SCHED) as srv:
        def client(chunk):
            ids = [srv.submit(*r) for r in chunk]
            return [srv.wait(rid, timeout=120, counts=True) for rid in ids]
        with cf.ThreadPoolExecutor(4) as pool:
            outs = list(pool.map(client, [reqs[i::4] for i in range(4)]))
        st = srv.stats()
    for i in range(4):
        for req, (sc, counts, _) in zip(reqs[i::4], outs[i]):
            check_against_oracle(hosts, req, sc, counts)
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["pending"] == 0
