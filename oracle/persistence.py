"""Persistence diagrams of a filtered complex and the bottleneck distance (§2).

A filtration function f on the simplices of Del(L) that is monotone (faces
never come after cofaces) induces the nested complexes Sigma_t = f^{-1}((-inf, t]).
Its persistence diagram dgm_k is the multiset of (birth, death) pairs of
k-dimensional homology classes (§2). Here it is computed by the standard
Z/2 column reduction of the boundary matrix, with simplices ordered by
(value, dimension, lexicographic vertex ids) so that faces precede cofaces
on ties, and with the clearing optimisation (a column whose index is already
a pivot is zero). Points on the diagonal (birth == death) are dropped.

The bottleneck distance d_B(D1, D2) = inf over bijections eta of
sup_p |p - eta(p)|_inf, the diagonal taken with infinite multiplicity (§2),
is computed exactly: binary search over the finite set of candidate costs
with a bipartite perfect-matching test at each candidate.
"""
from __future__ import annotations

import numpy as np

__all__ = ["filtration_order", "diagrams", "bottleneck"]


def filtration_order(simplices, values):
    """Global order of all simplices: list of (k, row) sorted by (value, k, vertex ids)."""
    entries = []
    for k, S in enumerate(simplices):
        S = np.asarray(S)
        v = np.asarray(values[k], dtype=np.float64)
        for r in range(S.shape[0]):
            entries.append((float(v[r]), k, tuple(int(a) for a in S[r]), r))
    entries.sort()
    return [(k, r) for (_, k, _, r) in entries], [e[0] for e in entries]


def diagrams(simplices, facets, values, max_dim: int | None = None):
    """dgm_0 .. dgm_{max_dim} as float64 arrays (n, 2); death = inf for essential classes."""
    K = len(simplices)
    if max_dim is None:
        max_dim = K - 1
    order, vals = filtration_order(simplices, values)
    pos = {kr: i for i, kr in enumerate(order)}
    for i, (k, r) in enumerate(order):
        for j in range(k + 1 if k > 0 else 0):
            if pos[(k - 1, int(facets[k][r][j]))] > i:
                raise ValueError("filtration is not monotone: a face enters after its coface")
    n = len(order)
    dims = [k for (k, _) in order]
    pivot_of = {}          # pivot row -> reduced column index
    reduced = {}
    cleared = set()
    # Process columns by decreasing dimension so that clearing applies (twist).
    for k in range(K - 1, 0, -1):
        for i in range(n):
            if dims[i] != k or i in cleared:
                continue
            kk, r = order[i]
            col = set(pos[(k - 1, int(facets[k][r][j]))] for j in range(k + 1))
            while col:
                p = max(col)
                other = pivot_of.get(p)
                if other is None:
                    break
                col ^= reduced[other]
            if col:
                p = max(col)
                pivot_of[p] = i
                reduced[i] = col
                cleared.add(p)
    dgms = [[] for _ in range(max_dim + 1)]
    paired = set()
    for p, i in pivot_of.items():
        paired.add(p)
        paired.add(i)
        k = dims[p]
        if k <= max_dim and vals[i] > vals[p]:
            dgms[k].append((vals[p], vals[i]))
    for i in range(n):
        if i in paired:
            continue
        if i in reduced:       # a non-zero reduced column is a death, never a birth
            continue
        k = dims[i]
        if k <= max_dim:
            dgms[k].append((vals[i], np.inf))
    return [np.array(sorted(d), dtype=np.float64).reshape(-1, 2) for d in dgms]


def _matching_exists(A, B, eps):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import maximum_bipartite_matching

    na, nb = A.shape[0], B.shape[0]
    n = na + nb
    rows, cols = [], []
    for i in range(na):
        for j in range(nb):
            if max(abs(A[i, 0] - B[j, 0]), abs(A[i, 1] - B[j, 1])) <= eps:
                rows.append(i)
                cols.append(j)
        if (A[i, 1] - A[i, 0]) / 2.0 <= eps:
            rows.append(i)
            cols.append(nb + i)               # A_i to its diagonal projection
    for j in range(nb):
        if (B[j, 1] - B[j, 0]) / 2.0 <= eps:
            rows.append(na + j)
            cols.append(j)                    # diagonal copy of B_j to B_j
        for i in range(na):
            rows.append(na + j)
            cols.append(nb + i)               # diagonal to diagonal is free
    if n == 0:
        return True
    M = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    match = maximum_bipartite_matching(M, perm_type="column")
    return bool(np.all(match >= 0))


def bottleneck(D1, D2) -> float:
    """Exact bottleneck distance between two diagrams given as (n, 2) arrays."""
    D1 = np.asarray(D1, dtype=np.float64).reshape(-1, 2)
    D2 = np.asarray(D2, dtype=np.float64).reshape(-1, 2)
    inf1, inf2 = D1[np.isinf(D1[:, 1])], D2[np.isinf(D2[:, 1])]
    if inf1.shape[0] != inf2.shape[0]:
        return float("inf")
    ess = float(np.max(np.abs(np.sort(inf1[:, 0]) - np.sort(inf2[:, 0])))) if inf1.shape[0] else 0.0
    A, B = D1[np.isfinite(D1[:, 1])], D2[np.isfinite(D2[:, 1])]
    cands = {0.0}
    for P in (A, B):
        cands.update(((P[:, 1] - P[:, 0]) / 2.0).tolist())
    for a in A:
        for b in B:
            cands.add(max(abs(a[0] - b[0]), abs(a[1] - b[1])))
    cands = np.array(sorted(cands))
    lo, hi = 0, len(cands) - 1
    while lo < hi:
        mid = (lo + hi) // 2
        if _matching_exists(A, B, cands[mid]):
            hi = mid
        else:
            lo = mid + 1
    return max(ess, float(cands[lo]))
