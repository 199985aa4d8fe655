"""Seeded graph generators producing undirected CSR graphs.

Layout of every graph returned here (the layout the library's loader takes):
  offsets : int64[n + 1], offsets[0] = 0, non-decreasing, offsets[n] = nnz
  nbrs    : uint32[nnz], row v = nbrs[offsets[v]:offsets[v + 1]], strictly
            increasing (sorted, no duplicates), no self-loops, symmetric
            (v in row u  <=>  u in row v), so nnz = 2m.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Graph:
    n: int
    offsets: np.ndarray  # int64[n+1]
    nbrs: np.ndarray  # uint32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    @property
    def degrees(self) -> np.ndarray:
        return np.diff(self.offsets)

    def row(self, v: int) -> np.ndarray:
        return self.nbrs[self.offsets[v]:self.offsets[v + 1]]

    def describe(self) -> dict:
        d = self.degrees
        return {
            "name": self.name,
            "n": int(self.n),
            "m": int(self.m),
            "nnz": int(self.nnz),
            "max_degree": int(d.max()) if self.n else 0,
            "isolated": int((d == 0).sum()),
        }


def csr_from_edges(n: int, u, v, name: str = "") -> Graph:
    """Symmetric sorted CSR from an undirected edge list.

    Self-loops are dropped and duplicate edges (in either orientation) merged.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = lo * n + hi
    key.sort()
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    lo = key // n
    hi = key % n
    # both orientations; keys are distinct, so sorting them orders the CSR
    both = np.concatenate([key, hi * n + lo])
    both.sort()
    src = both // n
    dst = both - src * n
    counts = np.bincount(src, minlength=n) if n else np.zeros(0, np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    return Graph(n, offsets, dst.astype(np.uint32), name)


def edges_of(g: Graph):
    """Canonical undirected edge list (u < v) in CSR order."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees)
    dst = g.nbrs.astype(np.int64)
    keep = src < dst
    return src[keep], dst[keep]


def all_edges(g: Graph) -> np.ndarray:
    """uint32[m, 2] array of canonical edges (u < v) in CSR order."""
    u, v = edges_of(g)
    return np.stack([u, v], axis=1).astype(np.uint32)


def relabel(g: Graph, seed: int) -> Graph:
    """Apply a seeded random permutation to the vertex ids."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(g.n).astype(np.int64)
    u, v = edges_of(g)
    return csr_from_edges(g.n, perm[u], perm[v], g.name)


def largest_component(g: Graph) -> Graph:
    """Induced subgraph on the largest connected component, ids compacted
    in increasing order of the old ids."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components

    if g.n == 0:
        return g
    mat = csr_matrix(
        (np.ones(g.nnz, dtype=np.int8), g.nbrs.astype(np.int64), g.offsets),
        shape=(g.n, g.n),
    )
    ncomp, labels = connected_components(mat, directed=False)
    if ncomp == 1:
        return g
    big = np.bincount(labels).argmax()
    keep = labels == big
    newid = np.full(g.n, -1, dtype=np.int64)
    newid[keep] = np.arange(int(keep.sum()))
    u, v = edges_of(g)
    sel = keep[u] & keep[v]
    return csr_from_edges(int(keep.sum()), newid[u[sel]], newid[v[sel]], g.name)


# --------------------------------------------------------------------------
# small exact cases
# --------------------------------------------------------------------------

def complete(n: int) -> Graph:
    u, v = np.triu_indices(n, 1)
    return csr_from_edges(n, u, v, f"K{n}")


def cycle(n: int) -> Graph:
    u = np.arange(n)
    return csr_from_edges(n, u, (u + 1) % n, f"C{n}")


def path(n: int) -> Graph:
    u = np.arange(n - 1)
    return csr_from_edges(n, u, u + 1, f"P{n}")


def diamond() -> Graph:
    """The 4-vertex, 5-edge graph of Fig. 1: A=0, B=1, C=2, D=3 with edges
    AB, AC, BC, BD, CD (deg A = deg D = 2, deg B = deg C = 3)."""
    u = [0, 0, 1, 1, 2]
    v = [1, 2, 2, 3, 3]
    return csr_from_edges(4, u, v, "diamond")


def prufer_tree(n: int, seed: int) -> Graph:
    """Uniform random labelled tree on n >= 2 vertices (Prufer decoding)."""
    rng = np.random.default_rng(seed)
    if n == 2:
        return csr_from_edges(2, [0], [1], "tree2")
    seq = rng.integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    for x in seq:
        degree[x] += 1
    us, vs = [], []
    for x in seq:
        leaf = int(np.flatnonzero(degree == 1)[0])
        us.append(leaf)
        vs.append(int(x))
        degree[leaf] -= 1
        degree[x] -= 1
    rest = np.flatnonzero(degree == 1)
    us.append(int(rest[0]))
    vs.append(int(rest[1]))
    return csr_from_edges(n, us, vs, f"tree{n}")


def _spanning_path(n: int, rng) -> tuple[np.ndarray, np.ndarray]:
    perm = rng.permutation(n)
    return perm[:-1], perm[1:]


def gnp_connected(n: int, p: float, seed: int) -> Graph:
    """G(n, p) plus a path over a seeded permutation (so it is connected)."""
    rng = np.random.default_rng(seed)
    iu, iv = np.triu_indices(n, 1)
    take = rng.random(iu.size) < p
    pu, pv = _spanning_path(n, rng)
    u = np.concatenate([iu[take], pu])
    v = np.concatenate([iv[take], pv])
    return csr_from_edges(n, u, v, f"gnp{n}")


def er_with_path(n: int, m: int, seed: int) -> Graph:
    """G(n, m): m distinct uniform random edges, plus a spanning path over a
    seeded permutation; duplicates merged (the tiny AESC workload)."""
    rng = np.random.default_rng(seed)
    chosen = np.zeros(0, dtype=np.int64)
    while chosen.size < m:
        a = rng.integers(0, n, size=2 * m)
        b = rng.integers(0, n, size=2 * m)
        keep = a != b
        key = np.minimum(a, b)[keep] * n + np.maximum(a, b)[keep]
        chosen = np.concatenate([chosen, key])
        _, first = np.unique(chosen, return_index=True)
        chosen = chosen[np.sort(first)]
    chosen = chosen[:m]
    pu, pv = _spanning_path(n, rng)
    u = np.concatenate([chosen // n, pu])
    v = np.concatenate([chosen % n, pv])
    return csr_from_edges(n, u, v, f"er{n}_{m}")


# --------------------------------------------------------------------------
# large synthetic stand-ins
# --------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0, relabel_seed: int | None = None) -> Graph:
    """R-MAT graph: 2^scale vertices, edge_factor * 2^scale generated edges,
    quadrant probabilities (a, b, c, 1 - a - b - c) at every level,
    symmetrised, self-loops and duplicates removed, ids randomly relabelled
    (R-MAT ids are otherwise ordered by expected degree)."""
    n = 1 << scale
    m = edge_factor * n
    rng = np.random.default_rng(seed)
    u = np.zeros(m, dtype=np.int64)
    v = np.zeros(m, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    for level in range(scale):
        r = rng.random(m, dtype=np.float64)
        ubit = r >= ab
        vbit = ((r >= a) & (r < ab)) | (r >= abc)
        u |= ubit.astype(np.int64) << level
        v |= vbit.astype(np.int64) << level
        del r, ubit, vbit
    perm = np.random.default_rng(seed + 1 if relabel_seed is None else relabel_seed)
    perm = perm.permutation(n).astype(np.int64)
    return csr_from_edges(n, perm[u], perm[v], f"rmat{scale}_ef{edge_factor}")


def chung_lu(n: int, mean_degree: float, exponent: float, seed: int,
             keep_lcc: bool = True) -> Graph:
    """Chung-Lu power-law graph: expected degrees w_i proportional to
    (i + 1)^(-1/(exponent - 1)), scaled to the mean degree and capped at
    sqrt(n * mean_degree); n * mean_degree / 2 edges with both endpoints drawn
    proportional to w; duplicates and self-loops removed; largest connected
    component kept; ids relabelled at random."""
    rng = np.random.default_rng(seed)
    w = (np.arange(n, dtype=np.float64) + 1.0) ** (-1.0 / (exponent - 1.0))
    w *= mean_degree * n / w.sum()
    w = np.minimum(w, np.sqrt(n * mean_degree))
    w *= mean_degree * n / w.sum()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    m = int(round(n * mean_degree / 2))
    u = np.searchsorted(cdf, rng.random(m), side="right")
    v = np.searchsorted(cdf, rng.random(m), side="right")
    u = np.minimum(u, n - 1)
    v = np.minimum(v, n - 1)
    g = csr_from_edges(n, u, v, f"chunglu{n}_{exponent}")
    if keep_lcc:
        g = largest_component(g)
    g = relabel(g, seed + 7)
    g.name = f"chunglu{n}_{exponent}"
    return g


def grid_deleted(rows: int, cols: int, delete_fraction: float, seed: int) -> Graph:
    """rows x cols 4-neighbour grid, a seeded fraction of edges deleted,
    largest connected component kept."""
    rng = np.random.default_rng(seed)
    idx = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    hu = idx[:, :-1].ravel()
    hv = idx[:, 1:].ravel()
    vu = idx[:-1, :].ravel()
    vv = idx[1:, :].ravel()
    u = np.concatenate([hu, vu])
    v = np.concatenate([hv, vv])
    keep = rng.random(u.size) >= delete_fraction
    g = csr_from_edges(rows * cols, u[keep], v[keep], f"grid{rows}x{cols}")
    g = largest_component(g)
    g.name = f"grid{rows}x{cols}"
    return g


def cached(key: str, builder) -> Graph:
    """builder() memoised on disk under $BQ_WORKLOAD_CACHE (default
    .workload_cache/ at the repository root), keyed by `key`."""
    import os

    root = os.environ.get("BQ_WORKLOAD_CACHE") or os.path.join(
        os.path.dirname(os.path.dirname(os.path.abspath(__file__))), ".workload_cache")
    path = os.path.join(root, key + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["offsets"], z["nbrs"], str(z["name"]))
    g = builder()
    try:
        os.makedirs(root, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, n=g.n, offsets=g.offsets, nbrs=g.nbrs, name=g.name)
        os.replace(tmp, path)
    except OSError:
        pass
    return g


def rmat20() -> Graph:
    """The random-walk benchmark graph: R-MAT scale 20, edge factor 16,
    (a, b, c) = (0.57, 0.19, 0.19), seed 20."""
    return cached("rmat20_ef16_s20", lambda: rmat(20, 16, 0.57, 0.19, 0.19, seed=20))


def batched_mix(count: int = 256, seed: int = 4, n_min: float = 1e3, n_max: float = 1e6):
    """The batched-AESC workload: `count` graphs with n log-uniform in
    [n_min, n_max] and mean degree uniform in [4, 16]; a third Erdos-Renyi
    (plus a spanning path), a third R-MAT (a, b, c = 0.57, 0.19, 0.19; scale
    round(log2 n), edge factor d/2; largest component), a third
    sqrt(n) x sqrt(n) grids with 10% of edges deleted (largest component).
    Returns [(graph, eps)] with eps drawn from {0.05, 0.1, 0.2}."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        d = float(rng.uniform(4.0, 16.0))
        eps = float(rng.choice([0.05, 0.1, 0.2]))
        kind = i % 3
        s = int(rng.integers(0, 2**31))
        key = f"mix{seed}_{i}_{kind}_{n}_{s}"
        if kind == 0:
            build = (lambda n=n, d=d, s=s: er_with_path(n, max(1, int(round(n * d / 2))), s))
        elif kind == 1:
            scale = max(4, int(round(np.log2(n))))
            build = (lambda scale=scale, d=d, s=s:
                     largest_component(rmat(scale, max(1, int(round(d / 2))), seed=s)))
        else:
            side = max(4, int(round(np.sqrt(n))))
            build = (lambda side=side, s=s: grid_deleted(side, side, 0.1, s))
        out.append((cached(key, build), eps))
    return out


def uniform_starts(g: Graph, n_walks: int, seed: int) -> np.ndarray:
    """uint32[n_walks] start vertices drawn uniformly over the vertices that
    have at least one neighbour (an isolated vertex has no walk to take)."""
    rng = np.random.default_rng(seed)
    live = np.flatnonzero(g.degrees > 0).astype(np.uint32)
    pick = rng.integers(0, live.size, size=n_walks)
    return live[pick]
