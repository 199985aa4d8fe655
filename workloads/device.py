"""Seeded graph generators that run on the GPU with torch (for inputs too
large to build quickly on the host: R-MAT scale 24, 4096 x 4096 grids).

They return CSR arrays on the device (int64 offsets[n+1], int32 nbrs[nnz],
rows sorted, symmetric, no self-loops or duplicates).  Results depend only on
the seed, the torch version and the device type.  Nothing here computes any
part of the random-walk method."""

from dataclasses import dataclass


@dataclass
class DeviceGraph:
    name: str
    n: int
    offsets: "object"  # torch.int64 [n + 1] on the device
    nbrs: "object"     # torch.int32 [nnz] on the device

    @property
    def nnz(self) -> int:
        return int(self.nbrs.numel())

    @property
    def m(self) -> int:
        return self.nnz // 2


def _csr_from_keys(torch, n: int, bits: int, u, v, name: str) -> DeviceGraph:
    """Symmetrise (u, v), drop self-loops and duplicates, build CSR."""
    keep = u != v
    u, v = u[keep], v[keep]
    keys = torch.cat([(u << bits) | v, (v << bits) | u])
    del u, v, keep
    keys = torch.unique(keys, sorted=True)
    rows = keys >> bits
    nbrs = (keys & ((1 << bits) - 1)).to(torch.int32)
    del keys
    counts = torch.bincount(rows, minlength=n)
    del rows
    offsets = torch.zeros(n + 1, dtype=torch.int64, device=nbrs.device)
    offsets[1:] = torch.cumsum(counts, 0)
    return DeviceGraph(name, n, offsets, nbrs)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0, device: str = "cuda") -> DeviceGraph:
    """R-MAT: 2^scale vertices, edge_factor * 2^scale generated edges, one
    quadrant draw per level with probabilities (a, b, c, 1 - a - b - c), ids
    relabelled by a seeded permutation, then symmetrised and deduplicated."""
    import torch
    n = 1 << scale
    m = edge_factor * n
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    u = torch.zeros(m, dtype=torch.int64, device=device)
    v = torch.zeros(m, dtype=torch.int64, device=device)
    ab, abc = a + b, a + b + c
    for level in range(scale):
        r = torch.rand(m, generator=gen, device=device)
        bit = 1 << (scale - 1 - level)
        u += (r >= ab).to(torch.int64) * bit
        v += (((r >= a) & (r < ab)) | (r >= abc)).to(torch.int64) * bit
        del r
    perm = torch.randperm(n, generator=gen, device=device)
    u = perm[u]
    v = perm[v]
    del perm
    return _csr_from_keys(torch, n, scale, u, v, f"rmat{scale}_ef{edge_factor}_s{seed}")


def grid(rows: int, cols: int, delete_fraction: float, seed: int, device: str = "cuda") -> DeviceGraph:
    """rows x cols 4-neighbour grid with a seeded fraction of its edges
    deleted (all vertices kept; ids row-major)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    idx = torch.arange(rows * cols, dtype=torch.int64, device=device).view(rows, cols)
    u = torch.cat([idx[:, :-1].reshape(-1), idx[:-1, :].reshape(-1)])
    v = torch.cat([idx[:, 1:].reshape(-1), idx[1:, :].reshape(-1)])
    keep = torch.rand(u.numel(), generator=gen, device=device) >= delete_fraction
    bits = max(1, (rows * cols - 1).bit_length())
    return _csr_from_keys(torch, rows * cols, bits, u[keep], v[keep], f"grid{rows}x{cols}_del{delete_fraction}")


def sample_edges(g, k: int, gen, device: str = "cuda"):
    """k edges drawn uniformly (with replacement) from the CSR entries of a
    device graph, as a host uint32 array of (u, v) pairs (either orientation:
    each undirected edge is two entries)."""
    import torch
    j = torch.randint(0, g.nnz, (k,), generator=gen, device=device)
    u = torch.searchsorted(g.offsets, j, right=True) - 1
    v = g.nbrs[j].to(torch.int64)
    return torch.stack([u, v], 1).to(torch.int32).cpu().numpy().view("uint32")
