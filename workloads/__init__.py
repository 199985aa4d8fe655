"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

This module holds no arithmetic of the estimation method: it only builds
graphs (symmetric CSR, sorted rows, no self-loops, no duplicate edges) and
draws start vertices.  Every generator takes an explicit seed and uses
numpy's PCG64 generator, so the same call gives the same graph on any
machine.

The graph families stand in for the paper's SNAP datasets (Table 1), which
are not available here: Erdos-Renyi with a spanning path, R-MAT, Chung-Lu
power-law graphs, 2-D grids with deleted edges, and the small exact cases
(complete graphs, cycles, random trees, the 4-vertex diamond of Fig. 1).
"""

from .graphs import (  # noqa: F401
    Graph,
    csr_from_edges,
    largest_component,
    relabel,
    complete,
    cycle,
    path,
    diamond,
    prufer_tree,
    gnp_connected,
    er_with_path,
    rmat,
    chung_lu,
    grid_deleted,
    uniform_starts,
    cached,
    rmat20,
    batched_mix,
    all_edges,
    edges_of,
)
