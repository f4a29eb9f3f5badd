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

__all__ = ["filtration_order", "persistence_pairs", "diagrams", "bottleneck", "bottleneck_within"]


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


def persistence_pairs(simplices, facets, values):
    """Persistence pairing of the filtration by the Z/2 column reduction.

    Returns (pairs, essential): pairs is a list of ((k, row), (k + 1, row')) with
    the simplex that creates a k-dimensional class and the one that kills it
    (zero-persistence pairs included); essential lists the (k, row) of the
    simplices whose classes never die. Simplices are ordered by (value,
    dimension, lexicographic vertex ids).
    """
    K = len(simplices)
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
    pairs = sorted((order[p], order[i]) for p, i in pivot_of.items())
    paired = set(pivot_of) | set(pivot_of.values())
    # a non-zero reduced column is a death, never a birth
    essential = [order[i] for i in range(n) if i not in paired and i not in reduced]
    return pairs, essential


def diagrams(simplices, facets, values, max_dim: int | None = None):
    """dgm_0 .. dgm_{max_dim} as float64 arrays (n, 2); death = inf for essential classes."""
    K = len(simplices)
    if max_dim is None:
        max_dim = K - 1
    pairs, essential = persistence_pairs(simplices, facets, values)
    val = lambda kr: float(np.asarray(values[kr[0]], dtype=np.float64)[kr[1]])  # noqa: E731
    dgms = [[] for _ in range(max_dim + 1)]
    for b, d in pairs:
        if b[0] <= max_dim and val(d) > val(b):
            dgms[b[0]].append((val(b), val(d)))
    for b in essential:
        if b[0] <= max_dim:
            dgms[b[0]].append((val(b), np.inf))
    return [np.array(sorted(d), dtype=np.float64).reshape(-1, 2) for d in dgms]


def _matching_exists(A, B, eps):
    """Perfect matching of A + diag(B) against B + diag(A) using only pairs within eps (L-inf)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import maximum_bipartite_matching

    na, nb = A.shape[0], B.shape[0]
    n = na + nb
    if n == 0:
        return True
    rows, cols = [], []
    if na and nb:
        cost = np.maximum(np.abs(A[:, None, 0] - B[None, :, 0]), np.abs(A[:, None, 1] - B[None, :, 1]))
        i, j = np.nonzero(cost <= eps)
        rows.append(i)
        cols.append(j)                            # A_i to B_j
    ia = np.nonzero((A[:, 1] - A[:, 0]) / 2.0 <= eps)[0]
    rows.append(ia)
    cols.append(nb + ia)                          # A_i to its diagonal projection
    jb = np.nonzero((B[:, 1] - B[:, 0]) / 2.0 <= eps)[0]
    rows.append(na + jb)
    cols.append(jb)                               # diagonal copy of B_j to B_j
    if na and nb:
        rr, cc = np.meshgrid(np.arange(nb), np.arange(na), indexing="ij")
        rows.append(na + rr.ravel())
        cols.append(nb + cc.ravel())              # diagonal to diagonal is free
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    M = coo_matrix((np.ones(r.shape[0]), (r, c)), shape=(n, n)).tocsr()
    match = maximum_bipartite_matching(M, perm_type="column")
    return bool(np.all(match >= 0))


def bottleneck_within(D1, D2, eps: float) -> bool:
    """True iff the bottleneck distance between two diagrams is at most eps (one matching test)."""
    D1 = np.asarray(D1, dtype=np.float64).reshape(-1, 2)
    D2 = np.asarray(D2, dtype=np.float64).reshape(-1, 2)
    inf1, inf2 = np.sort(D1[np.isinf(D1[:, 1]), 0]), np.sort(D2[np.isinf(D2[:, 1]), 0])
    if inf1.shape[0] != inf2.shape[0]:
        return False
    # essential points lie on a line: the sorted matching is a bottleneck-optimal one
    if inf1.shape[0] and np.max(np.abs(inf1 - inf2)) > eps:
        return False
    return _matching_exists(D1[np.isfinite(D1[:, 1])], D2[np.isfinite(D2[:, 1])], eps)


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
