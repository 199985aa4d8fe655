"""Batches of vertex-centric AESC estimates (bq_batch_create_shared): many
queries over graphs of uneven sizes and layouts, their vertex tasks in one
persistent launch.  Every query's counters and estimates must be
bit-identical to the oracle's vertex-centric estimator and to a single
bq_aesc_estimate_shared on it alone, also under CUDA-graph capture and
replay; a plan that outgrows the histograms sized at creation is refused."""

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
    """Graphs in three layouts (edge records, packed ids, plain CSR); queries
    on distinct-edge subsets (either orientation) and on all edges, with
    unequal tau and N at shared endpoints."""
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
            uv, uv_host = None, uv_all
        else:
            k = int(rng.integers(1, min(400, uv_all.shape[0]) + 1))
            uv_host = uv_all[rng.choice(uv_all.shape[0], k, replace=False)]
            if qi % 2:
                uv_host = uv_host[:, ::-1].copy()
            uv = u32(torch, uv_host)
        k = uv_host.shape[0]
        tau = rng.integers(1, 9, k).astype(np.uint32)
        nw = rng.integers(1, 700, k).astype(np.uint32)
        seed = int(rng.integers(0, 2**63))
        queries.append({"graph": graph, "seed": seed, "uv": uv, "tau": u32(torch, tau), "nwalks": u32(torch, nw)})
        host.append((g, seed, uv_host, tau, nw))
    return graphs, queries, host


@pytest.mark.parametrize("sampler,lanes", [(None, 2), (None, 8), ((1, 5, 32), 2)])
def test_shared_batch_matches_oracle_and_single(env, sampler, lanes):
    bq, torch = env
    rng = np.random.default_rng(13)
    graphs, queries, host = make_queries(bq, torch, rng)
    old = bq.get_tuning()
    bq.set_tuning(shared_lanes=lanes)  # kept by the batch from its creation
    batch = bq.Batch(queries, sampler=sampler, shared=True)
    bq.set_tuning(**old)
    assert batch.size() == sum(h[3].size for h in host)
    for _ in range(2):  # outputs are overwritten, not accumulated
        batch.run()
        bq.sync()
        for (counts, sc), (g, seed, uv, tau, nw), q in zip(batch.outputs, host, queries):
            oc, _, osc = oracle.aesc_shared_estimate(g, seed, uv, tau, nw, sampler=sampler)
            assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
            assert same_bits(sc.cpu().numpy(), osc)
    for (counts, sc), q in zip(batch.outputs, queries):
        c1, _, s1 = bq.aesc_estimate_shared(q["graph"], q["seed"], q["uv"], q["tau"], q["nwalks"], sampler=sampler)
        bq.sync()
        assert torch.equal(c1, counts) and torch.equal(s1.view(torch.int64), sc.view(torch.int64))
    batch.close()


def test_shared_batch_cuda_graph_capture_and_replay(env):
    bq, torch = env
    rng = np.random.default_rng(14)
    graphs, queries, host = make_queries(bq, torch, rng)
    batch = bq.Batch(queries, shared=True)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.run(stream)
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg, stream=stream):
        batch.run(stream)
    for c, _ in batch.outputs:
        c.zero_()
    for _ in range(2):
        cg.replay()
    torch.cuda.synchronize()
    bq.sync()
    for (counts, sc), (g, seed, uv, tau, nw) in zip(batch.outputs, host):
        oc, _, osc = oracle.aesc_shared_estimate(g, seed, uv, tau, nw)
        assert np.array_equal(counts.cpu().numpy().view(np.uint32), oc)
        assert same_bits(sc.cpu().numpy(), osc)
    # new plans of no larger tau between replays: the new results
    g, seed, uv, tau, nw = host[1]
    nw2 = (nw // 2 + 1).astype(np.uint32)
    queries[1]["nwalks"].copy_(u32(torch, nw2))
    cg.replay()
    torch.cuda.synchronize()
    bq.sync()
    oc, _, osc = oracle.aesc_shared_estimate(g, seed, uv, tau, nw2)
    assert np.array_equal(batch.outputs[1][0].cpu().numpy().view(np.uint32), oc)
    assert same_bits(batch.outputs[1][1].cpu().numpy(), osc)
    batch.close()


def test_shared_batch_plan_growth_and_repeats_are_refused(env):
    """A tau that grows past the largest tau a vertex had at creation gives
    NaN estimates and BQ_EINVAL for that query only; a repeated edge gives
    BQ_EINVAL; the other queries are unaffected."""
    bq, torch = env
    g = gnp_connected(80, 0.1, 5)
    graph = bq.Graph.from_csr(g)
    uv_all = all_edges(g)
    tau = np.full(uv_all.shape[0], 3, np.uint32)
    nw = np.full(uv_all.shape[0], 50, np.uint32)
    qa = {"graph": graph, "seed": 1, "uv": None, "tau": u32(torch, tau), "nwalks": u32(torch, nw)}
    qb = {"graph": graph, "seed": 2, "uv": u32(torch, uv_all[:30]), "tau": u32(torch, tau[:30]),
          "nwalks": u32(torch, nw[:30])}
    batch = bq.Batch([qa, qb], shared=True)
    batch.run()
    bq.sync()
    qa["tau"].copy_(u32(torch, np.full(uv_all.shape[0], 6, np.uint32)))
    batch.run()
    with pytest.raises(bq.BouquetError) as ei:
        bq.sync()
    assert ei.value.code == bq.EINVAL
    assert torch.isnan(batch.outputs[0][1]).all()
    oc, _, osc = oracle.aesc_shared_estimate(g, 2, uv_all[:30], tau[:30], nw[:30])
    assert np.array_equal(batch.outputs[1][0].cpu().numpy().view(np.uint32), oc)
    assert same_bits(batch.outputs[1][1].cpu().numpy(), osc)
    batch.close()
    rep = np.concatenate([uv_all[:5], uv_all[2:3, ::-1]])
    qc = {"graph": graph, "seed": 3, "uv": u32(torch, rep), "tau": u32(torch, np.full(6, 3, np.uint32)),
          "nwalks": u32(torch, np.full(6, 9, np.uint32))}
    batch = bq.Batch([qc], shared=True)
    batch.run()
    with pytest.raises(bq.BouquetError) as ei:
        bq.sync()
    assert ei.value.code == bq.EINVAL
    batch.close()
    graph.close()
