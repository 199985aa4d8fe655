"""Exact FP64 / integer references for spanning centrality (test infrastructure).

Each function follows a definition the paper states or relies on:
  * spanning_tree_count / sc_matrix_tree: SC(e) = 1 - T(G \\ e) / T(G)
    (Sec. 2.1), with T counted by Kirchhoff's matrix-tree theorem as the
    determinant of a reduced Laplacian, in exact integer arithmetic.
  * sc_pinv: SC(e) = R_eff(u, v) = (e_u - e_v)^T L^+ (e_u - e_v) for an
    unweighted connected graph (Kirchhoff; the exact quantity that the
    walk-based methods of Sec. 2.3 approximate).
  * spectrum: eigenvalues of D^-1/2 A D^-1/2, the matrix whose eigenpairs
    CalculateTau uses (Sec. 2.3).
  * truncated_series: the half-weighted walk series
      S_tau = sum_{l < tau} t_l + t_tau / 2,
      t_l = p_l(u,u)/d_u - p_l(u,v)/d_v - p_l(v,u)/d_u + p_l(v,v)/d_v,
    with p_l = P^l, P = D^-1 A (the expectation of the walk estimator,
    Alg. 1 at zero push depth).
  * expected_distinct_ratio: E(eta) = (beta/alpha)(1 - (1 - 1/beta)^alpha),
    Sec. 5.6.
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np


def adjacency(g) -> np.ndarray:
    A = np.zeros((g.n, g.n), dtype=np.float64)
    for v in range(g.n):
        A[v, g.row(v).astype(np.int64)] = 1.0
    return A


def laplacian(g) -> np.ndarray:
    A = adjacency(g)
    return np.diag(A.sum(axis=1)) - A


def _int_det(M) -> int:
    """Exact determinant of an integer matrix (fraction-free Bareiss)."""
    a = [[int(x) for x in row] for row in M]
    n = len(a)
    if n == 0:
        return 1
    sign = 1
    prev = 1
    for k in range(n - 1):
        if a[k][k] == 0:
            swap = next((r for r in range(k + 1, n) if a[r][k] != 0), None)
            if swap is None:
                return 0
            a[k], a[swap] = a[swap], a[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                a[i][j] = (a[i][j] * a[k][k] - a[i][k] * a[k][j]) // prev
        prev = a[k][k]
    return sign * a[n - 1][n - 1]


def spanning_tree_count(n: int, edges) -> int:
    """Number of spanning trees of the multigraph-free graph (n, edges)."""
    if n == 1:
        return 1
    L = [[0] * n for _ in range(n)]
    for u, v in edges:
        u, v = int(u), int(v)
        L[u][u] += 1
        L[v][v] += 1
        L[u][v] -= 1
        L[v][u] -= 1
    reduced = [row[1:] for row in L[1:]]
    return _int_det(reduced)


def sc_matrix_tree(g, uv) -> list[Fraction]:
    """Exact SC of each query edge by counting spanning trees with and
    without it (tiny graphs only)."""
    from workloads import edges_of

    eu, ev = edges_of(g)
    edges = list(zip(eu.tolist(), ev.tolist()))
    total = spanning_tree_count(g.n, edges)
    if total == 0:
        raise ValueError("graph is disconnected")
    out = []
    for a, b in np.asarray(uv).reshape(-1, 2).tolist():
        key = (min(a, b), max(a, b))
        rest = [e for e in edges if e != key]
        out.append(1 - Fraction(spanning_tree_count(g.n, rest), total))
    return out


def sc_pinv(g, uv) -> np.ndarray:
    """Effective resistance of each query edge from the dense FP64
    pseudoinverse of the Laplacian."""
    Lp = np.linalg.pinv(laplacian(g), hermitian=True)
    q = np.asarray(uv, dtype=np.int64).reshape(-1, 2)
    u, v = q[:, 0], q[:, 1]
    return Lp[u, u] + Lp[v, v] - 2.0 * Lp[u, v]


def is_bipartite(g) -> bool:
    color = np.full(g.n, -1, dtype=np.int64)
    for s in range(g.n):
        if color[s] >= 0:
            continue
        color[s] = 0
        stack = [s]
        while stack:
            x = stack.pop()
            for y in g.row(x).tolist():
                if color[y] < 0:
                    color[y] = 1 - color[x]
                    stack.append(y)
                elif color[y] == color[x]:
                    return False
    return True


def spectrum(g):
    """(eigenvalues ascending, lambda2, lambda_neg) of N = D^-1/2 A D^-1/2
    for a connected graph.  lambda2 is the second-largest eigenvalue;
    lambda_neg is the most negative eigenvalue once one eigenvalue -1 is
    removed for a bipartite graph (0.0 if none is left)."""
    d = g.degrees.astype(np.float64)
    A = adjacency(g)
    s = 1.0 / np.sqrt(d)
    N = A * s[:, None] * s[None, :]
    lam = np.linalg.eigvalsh(N)
    lambda2 = float(lam[-2]) if lam.size >= 2 else 0.0
    rest = lam[:-1]
    if is_bipartite(g) and rest.size:
        rest = rest[1:]  # drop the exact -1 (the smallest eigenvalue)
    lambda_neg = float(rest.min()) if rest.size else 0.0
    if lambda_neg > 0.0:
        lambda_neg = 0.0
    return lam, lambda2, lambda_neg


def eigen_embedding(g, omega: int):
    """The omega largest eigenvalues of N = D^-1/2 A D^-1/2 after the
    eigenvalue 1 (connected graph), their unit eigenvectors scaled by
    1/sqrt(d) as an (n, omega) array, the next eigenvalue (0.0 if none) and
    the most negative eigenvalue other than an exact -1 (as spectrum())."""
    d = g.degrees.astype(np.float64)
    A = adjacency(g)
    s = 1.0 / np.sqrt(d)
    lam, vec = np.linalg.eigh(A * s[:, None] * s[None, :])
    order = np.argsort(lam)[::-1][1:]  # drop the eigenvalue 1
    top = order[:omega]
    rest = float(lam[order[omega]]) if order.size > omega else 0.0
    _, _, lambda_neg = spectrum(g)
    return lam[top].copy(), vec[:, top] * s[:, None], rest, lambda_neg


def transition(g) -> np.ndarray:
    A = adjacency(g)
    return A / A.sum(axis=1, keepdims=True)


def series_terms(g, u: int, v: int, tau: int) -> np.ndarray:
    """t_0 .. t_tau of the walk series for edge (u, v)."""
    P = transition(g)
    d = g.degrees.astype(np.float64)
    terms = np.zeros(tau + 1)
    Pl = np.eye(g.n)
    for l in range(tau + 1):
        terms[l] = (Pl[u, u] / d[u] - Pl[u, v] / d[v]
                    - Pl[v, u] / d[u] + Pl[v, v] / d[v])
        Pl = Pl @ P
    return terms


def truncated_series(g, u: int, v: int, tau: int) -> float:
    t = series_terms(g, u, v, tau)
    return float(t[:tau].sum() + 0.5 * t[tau])


def walk_distribution(g, start: int, steps: int) -> np.ndarray:
    """Row `start` of P^steps: the exact law of a walk's position."""
    P = transition(g)
    x = np.zeros(g.n)
    x[start] = 1.0
    for _ in range(steps):
        x = x @ P
    return x


def expected_distinct_ratio(alpha: int, beta: int) -> float:
    """E(eta), Sec. 5.6: expected share of distinct items when alpha lanes
    each draw uniformly from beta items."""
    return (beta / alpha) * (1.0 - (1.0 - 1.0 / beta) ** alpha)
