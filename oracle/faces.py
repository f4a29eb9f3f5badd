"""Faces and facet incidence of a set of tetrahedra, by definition (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this.

The discretised complex of §4.1 admits a simplex only once all of its faces
have entered, so the filtration runs over every face of the triangulation of
L (§4). A face of a simplex is a subset of its vertices; the triangles are the
3-subsets of the tetrahedra and the edges the 2-subsets. The facet of simplex
sigma opposite vertex j is sigma without its j-th (ascending) vertex. This
module writes that out with Python sets and dictionaries, independently of
both the product's host builder and the device kernels.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np

__all__ = ["faces_by_definition", "facet_rows"]


def faces_by_definition(tets):
    """(triangles (n2, 3), edges (n1, 2)) as ascending rows in lexicographic order."""
    tris, edges = set(), set()
    for t in np.asarray(tets, dtype=np.int64).reshape(-1, 4).tolist():
        t = tuple(sorted(t))
        for f in combinations(t, 3):
            tris.add(f)
        for e in combinations(t, 2):
            edges.add(e)
    tri = np.array(sorted(tris), dtype=np.int64).reshape(-1, 3)
    edg = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    return tri, edg


def facet_rows(simplices, lower):
    """For each row of `simplices` (n, k+1) and each j, the row of `lower` equal to the
    simplex without its j-th vertex (KeyError if absent)."""
    where = {tuple(r): i for i, r in enumerate(np.asarray(lower, dtype=np.int64).tolist())}
    S = np.asarray(simplices, dtype=np.int64)
    out = np.empty(S.shape, dtype=np.int64)
    for i, r in enumerate(S.tolist()):
        for j in range(len(r)):
            out[i, j] = where[tuple(r[:j] + r[j + 1:])]
    return out
