"""Host-side simplicial complex of the landmarks: Del(L), its faces and facet incidence.

The paper triangulates the landmark set L on the host with CGAL or qhull (§4);
this is input to the flood computation and is not part of the GPU hot path.
Here scipy's Qhull wrapper produces the tetrahedra; every lower-dimensional
face is enumerated from them, and each k-simplex gets the ids of its k+1
facets so that the face-max pass (§4.1, discretised complex Flood_r(X,L,P): a
simplex enters only when all of its faces have) can propagate values upward.

Conventions (shared by the C ABI and the oracle):
  * simplices[k] is int32 of shape (n_k, k+1); vertex ids ascend inside a row
    and rows are in lexicographic order.
  * facets[k] (k >= 1) is int32 of shape (n_k, k+1); column j is the row index
    in simplices[k-1] of the facet obtained by dropping vertex j.
  * simplices[0] is arange(n_L)[:, None]; facets[0] is an empty (n_0, 1) array.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

__all__ = ["SimplexLists", "delaunay_complex", "complex_from_simplices"]


@dataclass
class SimplexLists:
    n_vertices: int
    simplices: list = field(default_factory=list)  # k -> (n_k, k+1) int32
    facets: list = field(default_factory=list)     # k -> (n_k, k+1) int32

    @property
    def counts(self) -> list:
        return [int(s.shape[0]) for s in self.simplices]

    @property
    def top_dim(self) -> int:
        return len(self.simplices) - 1

    def save(self, path: str) -> None:
        arrays = {f"s{k}": s for k, s in enumerate(self.simplices)}
        arrays.update({f"f{k}": f for k, f in enumerate(self.facets)})
        np.savez_compressed(path, n_vertices=self.n_vertices, **arrays)

    @staticmethod
    def load(path: str) -> "SimplexLists":
        z = np.load(path)
        K = sum(1 for k in z.files if k.startswith("s"))
        return SimplexLists(int(z["n_vertices"]),
                            [z[f"s{k}"] for k in range(K)],
                            [z[f"f{k}"] for k in range(K)])


def _row_keys(rows: np.ndarray, base: int) -> np.ndarray:
    rows = rows.astype(np.int64)
    k1 = rows.shape[1]
    if float(base) ** k1 >= 2.0 ** 62:
        raise ValueError("too many vertices for int64 simplex keys")
    key = np.zeros(rows.shape[0], dtype=np.int64)
    for j in range(k1):
        key = key * base + rows[:, j]
    return key


def _unique_rows(rows: np.ndarray, base: int) -> np.ndarray:
    rows = np.sort(rows, axis=1)
    key = _row_keys(rows, base)
    _, first = np.unique(key, return_index=True)   # np.unique sorts keys: lexicographic rows
    return rows[first].astype(np.int32)


def complex_from_simplices(maximal, n_vertices: int, top_dim: int | None = None) -> SimplexLists:
    """Close a set of simplices under taking faces and build facet incidence.

    `maximal` is a list of integer arrays, each (n, k+1) for some k (or one array).
    """
    if isinstance(maximal, np.ndarray):
        maximal = [maximal]
    maximal = [np.asarray(a, dtype=np.int64) for a in maximal if np.asarray(a).size]
    if top_dim is None:
        top_dim = max((a.shape[1] - 1 for a in maximal), default=0)
    base = max(int(n_vertices), 2)
    by_dim = {k: [] for k in range(top_dim + 1)}
    for a in maximal:
        k = a.shape[1] - 1
        for j in range(k, 0, -1):
            for cols in combinations(range(k + 1), j + 1):
                by_dim[j].append(a[:, cols])
    simplices = [np.arange(n_vertices, dtype=np.int32)[:, None]]
    for k in range(1, top_dim + 1):
        rows = np.concatenate(by_dim[k]) if by_dim[k] else np.zeros((0, k + 1), np.int64)
        simplices.append(_unique_rows(rows, base) if rows.shape[0] else rows.astype(np.int32))
    facets = [np.zeros((n_vertices, 1), dtype=np.int32)]
    for k in range(1, top_dim + 1):
        s = simplices[k].astype(np.int64)
        f = np.empty(s.shape, dtype=np.int32)
        if k == 1:
            f[:] = s[:, [1, 0]]        # dropping vertex j of an edge leaves the other vertex
        else:
            lower_keys = _row_keys(simplices[k - 1], base)
            for j in range(k + 1):
                sub = np.delete(s, j, axis=1)
                key = _row_keys(sub, base)
                pos = np.searchsorted(lower_keys, key)
                if s.shape[0] and (pos.max() >= lower_keys.shape[0] or
                                   np.any(lower_keys[pos] != key)):
                    raise ValueError("complex is not closed under faces")
                f[:, j] = pos
        facets.append(f)
    return SimplexLists(int(n_vertices), simplices, facets)


def delaunay_complex(L: np.ndarray, dim: int | None = None) -> SimplexLists:
    """Delaunay triangulation of the landmarks (scipy/Qhull, FP64 predicates).

    dim = 3 (default for (n, 3) input): tetrahedra and all their faces.
    dim = 2: the planar triangulation of (n, 2) landmarks, or of (n, 3)
    landmarks whose z coordinates are all 0 (a planar cloud embedded at z = 0,
    which the CUDA path evaluates exactly like a native planar one).
    (n, 4) and (n, 5) landmarks (ambient dimension 4 or 5, §5.3 scaling in d):
    the full-dimensional Delaunay simplices and all their faces, for the
    general-dimension path (flood_filtration_nd).
    """
    from scipy.spatial import Delaunay

    L = np.asarray(L, dtype=np.float64)
    if L.ndim != 2 or L.shape[1] not in (2, 3, 4, 5):
        raise ValueError("landmarks must be (n, d) with 2 <= d <= 5")
    if dim is None:
        dim = L.shape[1]
    if L.shape[1] in (4, 5):
        if dim != L.shape[1]:
            raise ValueError("(n, 4) and (n, 5) landmarks take dim = d")
        top = np.sort(Delaunay(L).simplices.astype(np.int64), axis=1)
        return complex_from_simplices([top], L.shape[0], top_dim=dim)
    if dim == 2:
        if L.shape[1] == 3:
            if np.any(L[:, 2] != 0.0):
                raise ValueError("dim = 2 needs z = 0 for every landmark")
            L = L[:, :2]
        tris = np.sort(Delaunay(L).simplices.astype(np.int64), axis=1)
        return complex_from_simplices([tris], L.shape[0], top_dim=2)
    if dim != 3 or L.shape[1] != 3:
        raise ValueError("dim must be 2, or 3 with (n, 3) landmarks")
    tri = Delaunay(L)
    tets = np.sort(tri.simplices.astype(np.int64), axis=1)
    return complex_from_simplices([tets], L.shape[0], top_dim=3)
