"""Flood values by definition, in FP64 (§4.1, Lemma 1; App. A.1 for the k-d tree).

The filtration value of a simplex sigma of Del(L) is the directed Hausdorff
distance from conv(sigma) to X (§4.1),

    f(sigma) = max_{p in conv sigma} min_{x in X} d(p, x),

which the paper replaces by the finite grid P_sigma of Lemma 1:

    f_P(sigma) = max_{p in P_sigma} min_{x in X} |p - x|.

P_sigma is the FULL grid, faces included: the discretised complex
Flood_r(X, L, P) admits sigma only when P_tau is flooded for every face tau of
sigma (§4.1), and P_tau ⊂ P_sigma, so the full-grid maximum already equals the
maximum over all faces. For a vertex, P_v = {v} and f(v) = d(v, X) (0 when
L ⊂ X; §3, after Definition 1). L need not be a subset of X (§3): everything
here is the definition, so it holds for any landmarks.

Nearest distances are taken either by brute force over all of X or with an
exact FP64 k-d tree (scipy's cKDTree), the paper's own CPU path (App. A.1).
X and L are promoted exactly from float32 to float64. Points may have any
number d of coordinates (the construction of §3-§4 does not depend on it;
Fig. 4c varies d); simplices then go up to dimension d.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .samples import barycentric, compositions, sample_points

__all__ = ["FloodResult", "nearest_distance", "flood_values", "ritter_ball", "KDIndex"]


class KDIndex:
    """Exact nearest-neighbour index over X (FP64)."""

    def __init__(self, X: np.ndarray, method: str = "kdtree"):
        self.X = np.asarray(X, dtype=np.float64)
        self.method = method
        self._tree = None
        if method == "kdtree":
            from scipy.spatial import cKDTree
            self._tree = cKDTree(self.X)
        elif method != "brute":
            raise ValueError(method)

    def query(self, Q: np.ndarray, k: int = 1):
        """(dist, idx) of the nearest point(s); brute force breaks ties to the lowest index."""
        Q = np.asarray(Q, dtype=np.float64).reshape(-1, self.X.shape[1])
        if self.method == "kdtree":
            d, i = self._tree.query(Q, k=k, workers=-1)
            return d, i.astype(np.int64)
        return _brute_query(Q, self.X, k)


def _brute_query(Q, X, k=1):
    n = Q.shape[0]
    out_d = np.empty((n, k)) if k > 1 else np.empty(n)
    out_i = np.empty((n, k), dtype=np.int64) if k > 1 else np.empty(n, dtype=np.int64)
    chunk = max(1, 4_000_000 // max(1, X.shape[0]))
    for s in range(0, n, chunk):
        q = Q[s:s + chunk]
        diff = q[:, None, :] - X[None, :, :]
        d2 = (diff * diff).sum(axis=2)
        if k == 1:
            i = np.argmin(d2, axis=1)                  # first minimum: lowest index
            out_i[s:s + chunk] = i
            out_d[s:s + chunk] = np.sqrt(d2[np.arange(q.shape[0]), i])
        else:
            i = np.argsort(d2, axis=1, kind="stable")[:, :k]
            out_i[s:s + chunk] = i
            out_d[s:s + chunk] = np.sqrt(np.take_along_axis(d2, i, axis=1))
    return out_d, out_i


def nearest_distance(Q: np.ndarray, X: np.ndarray, method: str = "brute"):
    """min_{x in X} |q - x| for each row q of Q, with the arg-min index."""
    return KDIndex(X, method).query(Q)


@dataclass
class FloodResult:
    values: list          # k -> float64 (n_k,): f_P(sigma)
    argmax_sample: list   # k -> int64 (n_k,): rank of the attaining sample in the full grid
    argmin_point: list    # k -> int64 (n_k,): index in X of the nearest point of that sample
    simplex_ids: list     # k -> int64 (n_k,): which rows of simplices[k] were evaluated


def _vertex_coords(L, simplices_k, ids):
    return np.asarray(L, dtype=np.float64)[simplices_k[ids].astype(np.int64)]   # (n, k+1, d)


def flood_values(X, L, simplices, m: int, method: str = "brute", index: KDIndex | None = None,
                 subset=None, max_batch_samples: int = 2_000_000) -> FloodResult:
    """f_P(sigma) for every simplex (or the rows listed in subset[k]) of each dimension.

    simplices: list of int arrays, k -> (n_k, k+1), rows index L.
    """
    if m < 1:
        raise ValueError("m must be >= 1")
    if index is None:
        index = KDIndex(X, method)
    values, amax, amin, sids = [], [], [], []
    for k, S in enumerate(simplices):
        S = np.asarray(S)
        ids = np.arange(S.shape[0]) if subset is None or subset[k] is None else np.asarray(subset[k], np.int64)
        comps = compositions(m, k) if k > 0 else np.ones((1, 1), dtype=np.int64) * m
        F = comps.shape[0]
        val = np.empty(ids.shape[0])
        am = np.empty(ids.shape[0], dtype=np.int64)
        an = np.empty(ids.shape[0], dtype=np.int64)
        step = max(1, max_batch_samples // F)
        for s in range(0, ids.shape[0], step):
            sel = ids[s:s + step]
            V = _vertex_coords(L, S, sel)                          # (b, k+1, d)
            P = sample_points(V, comps, m)                         # (b, F, d): sum_j lambda_j v_j
            d, i = index.query(P.reshape(-1, P.shape[-1]))
            d = d.reshape(sel.shape[0], F)
            i = i.reshape(sel.shape[0], F)
            j = np.argmax(d, axis=1)                               # first maximum: lowest sample rank
            val[s:s + step] = d[np.arange(sel.shape[0]), j]
            am[s:s + step] = j
            an[s:s + step] = i[np.arange(sel.shape[0]), j]
        values.append(val)
        amax.append(am)
        amin.append(an)
        sids.append(ids)
    return FloodResult(values, amax, amin, sids)


def ritter_ball(V: np.ndarray):
    """Enclosing ball of Lemma 2's masking step (§4.2, Ritter-style variant).

    c is the midpoint of the longest edge of sigma and r = max_i d(c, v_i);
    the mask radius is sqrt(2) r for k >= 2 and r (half the edge length) for an edge.
    Returns (c, r, mask_radius).
    """
    V = np.asarray(V, dtype=np.float64)
    k1 = V.shape[0]
    best, pair = -1.0, (0, 0)
    for a in range(k1):
        for b in range(a + 1, k1):
            d = np.linalg.norm(V[a] - V[b])
            if d > best:
                best, pair = d, (a, b)
    c = 0.5 * (V[pair[0]] + V[pair[1]])
    r = float(np.max(np.linalg.norm(V - c, axis=1)))
    return c, r, (r if k1 == 2 else np.sqrt(2.0) * r)
