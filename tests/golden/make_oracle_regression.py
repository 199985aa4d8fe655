"""Writes oracle_regression.txt: sha256 digests of the CPU oracle's outputs on
small seeded inputs (walk visits and paths for three samplers, AESC counters
and estimates, push-phase accumulators at depths up to 0, 1 and 3, vertex-centric
counters, pilot moments, plans).  It calls only the oracle and the seeded input
generators; the fixture makes any later change to the oracle's arithmetic show
up as a change of this file.

    python tests/golden/make_oracle_regression.py
"""

import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import all_edges, diamond, er_with_path, gnp_connected, uniform_starts  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_regression.txt")


def digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:32]


def rows():
    out = []
    for g in (diamond(), gnp_connected(12, 0.4, 5), er_with_path(60, 150, 3)):
        starts = uniform_starts(g, 500, 9)
        for name, smp in (("ind", None), ("coupled", (1, 5, 8)), ("saba", (2, 0, 1))):
            vis, paths = oracle.walk_batch(g, 11, starts, 9, sampler=smp, include_start=True, want_paths=True)
            out.append((f"{g.name} walks {name}", digest(vis, paths)))
        uv = all_edges(g)
        tau, nw = oracle.plan_scheduled(g, uv, 0.1, 2.0, 2, 64, 9.0, 32)
        out.append((f"{g.name} plan scheduled", digest(tau, nw)))
        nw = (nw // 4 + 1).astype(np.uint32)
        counts, sc = oracle.aesc_estimate(g, 13, uv, tau, nw)
        out.append((f"{g.name} aesc", digest(counts, sc)))
        counts, sc = oracle.aesc_estimate(g, 13, uv, tau, nw, (1, 8, 32))
        out.append((f"{g.name} aesc coupled", digest(counts, sc)))
        for pm in (0, 1, 3):
            depth, acc, psc = oracle.aesc_push_estimate(g, 13, uv, tau, (nw * 20).astype(np.uint32), pm)
            out.append((f"{g.name} push max {pm}", digest(depth, acc, psc)))
        scounts, nused, ssc = oracle.aesc_shared_estimate(g, 13, uv, tau, nw)
        out.append((f"{g.name} shared", digest(scounts, nused, ssc)))
        ptau, pnw, mo, var = oracle.plan_pilot(g, 13, uv, 0.1, 2.0, 2, 64, 32, 50)
        out.append((f"{g.name} pilot", digest(ptau, pnw, mo, var)))
    return out


def main():
    with open(OUT, "w") as fh:
        fh.write("# sha256 (first 32 hex digits) of the CPU oracle's outputs on seeded inputs,\n")
        fh.write("# written by make_oracle_regression.py (which calls only the oracle).\n")
        fh.write("# Columns: case | digest\n")
        for name, d in rows():
            fh.write(f"{name} | {d}\n")


if __name__ == "__main__":
    main()
