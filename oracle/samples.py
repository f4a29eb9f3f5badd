"""Barycentric sample grid P_sigma of Lemma 1 (§4.1).

For a k-simplex sigma = {v_0, ..., v_k} and resolution m, Lemma 1 defines

    P_sigma = { sum_i lambda_i v_i : sum_i lambda_i = 1, m * lambda_i in N },

i.e. one point per composition (c_0, ..., c_k) of m into k+1 non-negative
parts, lambda_i = c_i / m. An edge carries m+1 grid points ("m+1 points per
edge"; 20 points per edge gives 210 points on a triangle and 1540 on a
tetrahedron, §5.3). Compositions are enumerated in lexicographic order of
(c_0, ..., c_k); a sample's id is its rank in that order. The interior grid
(all c_i >= 1) is the subset used by the CUDA path, whose sample ids are the
ranks among interior compositions, also lexicographic.
"""
from __future__ import annotations

from math import comb

import numpy as np

__all__ = ["compositions", "interior_compositions", "full_grid_count", "interior_count",
           "sample_points", "barycentric"]


def compositions(m: int, k: int, lo: int = 0) -> np.ndarray:
    """All (c_0..c_k) with c_i >= lo and sum m, lexicographic, as int64 (n, k+1)."""
    out = []

    def rec(prefix, remaining, parts_left):
        if parts_left == 1:
            if remaining >= lo:
                out.append(prefix + [remaining])
            return
        for c in range(lo, remaining - lo * (parts_left - 1) + 1):
            rec(prefix + [c], remaining - c, parts_left - 1)

    rec([], m, k + 1)
    return np.array(out, dtype=np.int64).reshape(-1, k + 1)


def interior_compositions(m: int, k: int) -> np.ndarray:
    """Compositions with every part >= 1 (points in the relative interior)."""
    return compositions(m, k, lo=1)


def full_grid_count(m: int, k: int) -> int:
    return comb(m + k, k)


def interior_count(m: int, k: int) -> int:
    return comb(m - 1, k) if m >= 1 else 0


def barycentric(comps: np.ndarray, m: int) -> np.ndarray:
    """lambda_i = c_i / m (Lemma 1), FP64."""
    return np.asarray(comps, dtype=np.float64) / float(m)


def sample_points(V: np.ndarray, comps: np.ndarray, m: int) -> np.ndarray:
    """p = sum_i lambda_i v_i in FP64.

    V is (k+1, d) for one simplex -> (n, d), or (b, k+1, d) for a batch -> (b, n, d).
    """
    lam = barycentric(comps, m)
    V = np.asarray(V, dtype=np.float64)
    if V.ndim == 2:
        return lam @ V
    return np.einsum("fj,bjd->bfd", lam, V)
