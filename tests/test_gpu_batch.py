"""AESC batches: many queries over graphs of uneven sizes and layouts in one
persistent counting launch.  Every query's counters and estimates must be
bit-identical to the oracle's (and so to a single bq_aesc_estimate), also
when the batch is captured in a CUDA graph and replayed."""

import numpy as np
import pytest

import oracle
from workloads import all_edges, er_with_path, gnp_connected, grid_deleted, rmat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq
    assert torch.cuda.is_available()
    return bq, torch


def u32(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def same_bits(a, b):
    return np.array_equal(np.asarray(a, np.float64).view(np.uint64), np.asarray(b, np.float64).view(np.uint64))


def make_queries(bq, torch, rng):
    """Graphs in three layouts (edge records, packed ids, plain CSR), queries
    on subsets (either orientation) and on all edges."""
    specs = [(gnp_connected(60, 0.1, 1), 1), (rmat(12, 8, seed=2), 5), (grid_deleted(20, 20, 0.1, 3), 0),
             (er_with_path(1000, 5000, 1), 1), (gnp_connected(200, 0.05, 9), 5)]
    old = bq.get_tuning()
    graphs, queries, host = [], [], []
    try:
        for g, layout in specs:
            bq.set_tuning(layout=layout)
            graphs.append((g, bq.Graph.from_csr(g)))
    finally:
        bq.set_tuning(**old)
    for qi in range(9):
        g, graph = graphs[qi % len(graphs)]
        uv_all = all_edges(g)
        if qi % 3 == 0:
            uv = None
            k = uv_all.shape[0]
            uv_host = uv_all
        else:
            k = int(rng.integers(1, min(300, uv_all.shape[0]) + 1))
            uv_host = uv_all[rng.choice(uv_all.shape[0], k, replace=False)]
            if qi % 2:
                uv_host = uv_host[:, ::-1].copy()
            uv = u32(torch, uv_host)
        tau = rng.integers(1, 9, k).astype(np.uint32)
        nw = rng.integers(1, 700, k).astype(np.uint32)
        seed = int(rng.integers(0, 2**63))
        queries.append({"graph": graph, "seed": seed, "uv": uv, "tau": u32(torch, tau),
                        "nwalks": u32(torch, nw)})
        host.append((g, seed, uv_host, tau, nw))
    return graphs, queries, host


@pytest.mark.parametrize("sampler", [None, (1, 5, 32)])
def test_batch_matches_oracle_and_single(env, sampler):
    bq, torch = env
    rng = np.random.default_rng(3)
    graphs, queries, host = make_queries(bq, torch, rng)
    batch = bq.Batch(queries, sampler=sampler)
    assert batch.size() == sum(h[3].size for h in host)
    batch.run()
    bq.sync()
    for (counts, sc), (g, seed, uv, tau, nw), q in zip(batch.outputs, host, queries):
        oc, osc = oracle.aesc_estimate(g, seed, uv, tau, nw, sampler=sampler)
        assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
        assert same_bits(sc.cpu().numpy(), osc)
        c1, s1 = bq.aesc_estimate(q["graph"], seed, q["uv"], q["tau"], q["nwalks"], sampler=sampler)
        bq.sync()
        assert np.array_equal(c1.cpu().numpy().view(np.uint32), oc)
    # running again gives the same results (outputs are overwritten, not accumulated)
    batch.run()
    bq.sync()
    g, seed, uv, tau, nw = host[0]
    oc, _ = oracle.aesc_estimate(g, seed, uv, tau, nw, sampler=sampler)
    assert np.array_equal(batch.outputs[0][0].cpu().numpy().view(np.uint32), oc)
    batch.close()


def test_batch_cuda_graph_capture_and_replay(env):
    bq, torch = env
    rng = np.random.default_rng(8)
    graphs, queries, host = make_queries(bq, torch, rng)
    batch = bq.Batch(queries)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run()  # warm-up outside the capture (kernel attributes, occupancy)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        batch.run()
    for out in batch.outputs:
        out[0].zero_()
        out[1].zero_()
    cg.replay()
    torch.cuda.synchronize()
    bq.sync()
    for (counts, sc), (g, seed, uv, tau, nw) in zip(batch.outputs, host):
        oc, osc = oracle.aesc_estimate(g, seed, uv, tau, nw)
        assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
        assert same_bits(sc.cpu().numpy(), osc)
    # new plans written into the same device buffers are picked up by a replay
    g, seed, uv, tau, nw = host[1]
    queries[1]["tau"].copy_(u32(torch, np.minimum(tau + 1, 9)))
    cg.replay()
    torch.cuda.synchronize()
    oc, _ = oracle.aesc_estimate(g, seed, uv, np.minimum(tau + 1, 9), nw)
    assert np.array_equal(batch.outputs[1][0].cpu().numpy().view(np.uint32), oc)
    batch.close()


def test_autotuners_pick_a_candidate_and_change_nothing(env):
    bq, torch = env
    from workloads import uniform_starts
    old = bq.get_tuning()
    try:
        g = rmat(12, 8, seed=2)
        graph = bq.Graph.from_csr(g)
        starts = uniform_starts(g, 50000, 1)
        st = u32(torch, starts)
        best, ms = bq.autotune_walks(graph, 4, st, 16)
        assert best in (1, 2, 4) and len(ms) == 3 and min(ms) > 0
        assert bq.get_tuning()["walk_lanes"] == best
        vis = bq.walk_batch(graph, 4, st, 16)
        bq.sync()
        assert np.array_equal(vis.cpu().numpy().view(np.uint32), oracle.walk_batch(g, 4, starts, 16))
        rng = np.random.default_rng(5)
        graphs, queries, host = make_queries(bq, torch, rng)
        best, ms = bq.autotune_aesc(queries)
        assert best in (2, 4, 8) and bq.get_tuning()["aesc_lanes"] == best
        batch = bq.Batch(queries)
        batch.run()
        bq.sync()
        for (counts, _), (hg, seed, uv, tau, nw) in zip(batch.outputs, host):
            oc, _ = oracle.aesc_estimate(hg, seed, uv, tau, nw)
            assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
        batch.close()
    finally:
        bq.set_tuning(**old)


def test_batch_invalid_pairs(env):
    bq, torch = env
    from workloads import cycle
    g = cycle(10)
    graph = bq.Graph.from_csr(g)
    uv = np.array([[0, 1], [0, 5], [3, 4]], np.uint32)
    tau = np.array([4, 4, 0], np.uint32)
    nw = np.array([50, 50, 50], np.uint32)
    batch = bq.Batch([{"graph": graph, "seed": 1, "uv": u32(torch, uv), "tau": u32(torch, tau),
                       "nwalks": u32(torch, nw)}])
    batch.run()
    with pytest.raises(bq.BouquetError):
        bq.sync()
    sc = batch.outputs[0][1].cpu().numpy()
    assert np.isfinite(sc[0]) and np.isnan(sc[1]) and np.isnan(sc[2])
    _, osc = oracle.aesc_estimate(g, 1, uv[:1], tau[:1], nw[:1])
    assert same_bits(sc[:1], osc)
    batch.close()
    with pytest.raises(bq.BouquetError):
        bq.Batch([])
