"""Input generators: the graphs they return are valid symmetric CSR with the
structure their recipe states (run on the CPU; the torch generators accept
device="cpu")."""

import numpy as np
import pytest

from workloads import chung_lu, grid_deleted, rmat
from workloads import device as dev


def check_csr(n, offsets, nbrs):
    offsets = np.asarray(offsets, np.int64)
    nbrs = np.asarray(nbrs).astype(np.int64)
    assert offsets.size == n + 1 and offsets[0] == 0 and offsets[-1] == nbrs.size
    assert np.all(np.diff(offsets) >= 0)
    rows = np.repeat(np.arange(n), np.diff(offsets))
    assert np.all((nbrs >= 0) & (nbrs < n)) and not np.any(rows == nbrs)
    keys = rows * n + nbrs
    assert np.all(np.diff(keys) > 0)  # rows sorted, no duplicates
    assert np.array_equal(np.sort(nbrs * n + rows), keys)  # symmetric


@pytest.mark.parametrize("g", [rmat(10, 8, seed=3), chung_lu(3000, 6.0, 2.3, 1), grid_deleted(15, 17, 0.1, 2)],
                         ids=["rmat", "chung_lu", "grid"])
def test_host_generators_valid(g):
    check_csr(g.n, g.offsets, g.nbrs)


def test_device_rmat_valid_and_seeded():
    import torch
    a = dev.rmat(11, 8, seed=4, device="cpu")
    check_csr(a.n, a.offsets.numpy(), a.nbrs.numpy())
    b = dev.rmat(11, 8, seed=4, device="cpu")
    assert torch.equal(a.nbrs, b.nbrs) and torch.equal(a.offsets, b.offsets)
    c = dev.rmat(11, 8, seed=5, device="cpu")
    assert not torch.equal(a.offsets, c.offsets)
    # skew: the top 1% of vertices hold far more than 1% of the edge ends
    deg = np.diff(a.offsets.numpy())
    top = np.sort(deg)[::-1][: a.n // 100].sum()
    assert top > 0.1 * deg.sum()


def test_device_grid_structure():
    full = dev.grid(20, 30, 0.0, 1, device="cpu")
    check_csr(full.n, full.offsets.numpy(), full.nbrs.numpy())
    assert full.m == 2 * 20 * 30 - 20 - 30
    deg = np.diff(full.offsets.numpy()).reshape(20, 30)
    assert deg[1:-1, 1:-1].min() == 4 and deg[0, 0] == 2 and deg[0, 5] == 3
    cut = dev.grid(40, 40, 0.05, 7, device="cpu")
    check_csr(cut.n, cut.offsets.numpy(), cut.nbrs.numpy())
    full_m = 2 * 40 * 40 - 80
    assert 0.9 * full_m < cut.m < full_m


def test_device_edge_sampler():
    import torch
    g = dev.rmat(9, 8, seed=1, device="cpu")
    gen = torch.Generator(device="cpu")
    gen.manual_seed(3)
    uv = dev.sample_edges(g, 2000, gen, device="cpu")
    off, nb = g.offsets.numpy(), g.nbrs.numpy()
    for u, v in uv[:200]:
        assert v in nb[off[u]:off[u + 1]]
    # both orientations occur
    assert np.any(uv[:, 0] < uv[:, 1]) and np.any(uv[:, 0] > uv[:, 1])
