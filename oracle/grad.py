"""Derivatives of F = sum_sigma gamma_sigma f_P(sigma) with respect to X and L (FP64).

The paper does not differentiate the filtration; this is our derivation of
the value definition of §4.1. f_P(sigma) = |p* - x*| where p* = sum_j lambda_j v_j
is the attaining grid sample (Lemma 1) and x* its nearest point of X. On a
smooth piece (unique attaining pair, f > 0):

    d f / d x*   = (x* - p*) / f
    d f / d v_j  = lambda_j (p* - x*) / f

and f = 0 contributes a zero subgradient. A vertex value f(v) = d(v, X) is
the case p* = v (its grid is the vertex itself): 0 when v is a point of X,
otherwise |v - x*| with the same two derivatives. X and L are independent
inputs: moving a landmark does not move its copy in X, and vice versa.

`finite_difference` evaluates (F(theta+h) - F(theta-h)) / 2h for single
coordinates with the simplex lists held fixed, recomputing only the simplices
whose values can change, and flags probes where the attaining (sample, point)
pair of an affected simplex changes within +-h ("kinks").
"""
from __future__ import annotations

import numpy as np

from .flood import FloodResult, KDIndex, flood_values
from .samples import barycentric, compositions, sample_points

__all__ = ["analytic_gradient", "finite_difference", "total"]


def total(result: FloodResult, gamma) -> float:
    """F = sum over k >= 0 of sum_sigma gamma_sigma f(sigma) (vertices included)."""
    return float(sum(np.dot(np.asarray(gamma[k], np.float64)[result.simplex_ids[k]], result.values[k])
                     for k in range(len(result.values))))


def analytic_gradient(X, L, simplices, m, gamma, result: FloodResult | None = None,
                      method: str = "kdtree"):
    """(dX (N,3), dL (n_L,3)) in FP64."""
    X64 = np.asarray(X, dtype=np.float64)
    L64 = np.asarray(L, dtype=np.float64)
    if result is None:
        result = flood_values(X, L, simplices, m, method=method)
    dX = np.zeros_like(X64)
    dL = np.zeros_like(L64)
    for k in range(len(simplices)):
        S = np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1)[result.simplex_ids[k]]
        if S.shape[0] == 0:
            continue
        g = np.asarray(gamma[k], dtype=np.float64)[result.simplex_ids[k]]
        lam = barycentric(compositions(m, k), m)[result.argmax_sample[k]]               # (n, k+1)
        V = L64[S]                                                                      # (n, k+1, 3)
        p = np.einsum("nj,njd->nd", lam, V)
        xi = result.argmin_point[k]
        x = X64[xi]
        f = np.linalg.norm(p - x, axis=1)
        ok = f > 0
        u = np.zeros_like(p)
        u[ok] = (p[ok] - x[ok]) / f[ok, None]
        np.add.at(dX, xi[ok], -(g[ok, None] * u[ok]))
        for j in range(k + 1):
            np.add.at(dL, S[ok, j], g[ok, None] * lam[ok, j, None] * u[ok])
    return dX, dL


class _AllSamples:
    """Every full-grid sample of every simplex (vertices included) with its two nearest points of X."""

    def __init__(self, X, L, simplices, m, index: KDIndex):
        self.k_of, self.rows, self.P, self.owner = [], [], [], []
        L64 = np.asarray(L, dtype=np.float64)
        dv, _ = index.query(L64)                                                     # d(v_j, X)
        self.ranges = {}
        start = 0
        Ps, boxes_lo, boxes_hi, ubs = [], [], [], []
        for k in range(len(simplices)):
            S = np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1)
            comps = compositions(m, k)
            V = L64[S]
            P = sample_points(V, comps, m)                                          # (n, F, 3)
            # u_p = min_j (|p - v_j| + d(v_j, X)) bounds d(p, X) (triangle inequality)
            u = np.min(np.linalg.norm(P[:, :, None, :] - V[:, None, :, :], axis=3) + dv[S][:, None, :], axis=2)
            self.ranges[k] = (start, S.shape[0], comps.shape[0])
            start += S.shape[0] * comps.shape[0]
            Ps.append(P.reshape(-1, 3))
            boxes_lo.append(P.min(axis=1) - u.max(axis=1)[:, None])
            boxes_hi.append(P.max(axis=1) + u.max(axis=1)[:, None])
        self.P = np.concatenate(Ps)
        self.box_lo = boxes_lo
        self.box_hi = boxes_hi
        d, i = index.query(self.P, k=2)
        self.d1, self.d2 = d[:, 0], d[:, 1]
        self.i1, self.i2 = i[:, 0], i[:, 1]

    def block(self, k, sid):
        s0, n, F = self.ranges[k]
        a = s0 + sid * F
        return slice(a, a + F)


def finite_difference(X, L, simplices, m, gamma, probes, h: float = 1e-3,
                      method: str = "kdtree", index: KDIndex | None = None, cache=None):
    """Central differences of F for probes [(which in {'X','L'}, row, col), ...].

    Returns (fd float64[n], kink bool[n], cache). The cache holds the sample
    table and may be passed back in for further probes on the same inputs.
    """
    X64 = np.asarray(X, dtype=np.float64)
    L64 = np.asarray(L, dtype=np.float64)
    if index is None:
        index = KDIndex(X64, method)
    if cache is None:
        cache = _AllSamples(X64, L64, simplices, m, index)
    A = cache
    fd = np.zeros(len(probes))
    kink = np.zeros(len(probes), dtype=bool)
    for t, (which, row, col) in enumerate(probes):
        plus = minus = 0.0
        changed = False
        if which == "L":
            for k in range(len(simplices)):
                S = np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1)
                sids = np.nonzero((S == row).any(axis=1))[0]
                if sids.size == 0:
                    continue
                g = np.asarray(gamma[k], dtype=np.float64)[sids]
                base = flood_values(X64, L64, [np.zeros((0, j + 1), np.int64) for j in range(k)] + [S],
                                    m, index=index, subset=[None] * k + [sids])
                vals = []
                for sgn in (+1.0, -1.0):
                    Lp = L64.copy()
                    Lp[row, col] += sgn * h
                    r = flood_values(X64, Lp, [np.zeros((0, j + 1), np.int64) for j in range(k)] + [S],
                                     m, index=index, subset=[None] * k + [sids])
                    vals.append(np.dot(g, r.values[k]))
                    changed |= bool(np.any(r.argmax_sample[k] != base.argmax_sample[k]) or
                                    np.any(r.argmin_point[k] != base.argmin_point[k]))
                plus += vals[0]
                minus += vals[1]
        else:
            x0 = X64[row]
            for k in range(len(simplices)):
                lo, hi = A.box_lo[k], A.box_hi[k]
                near = np.nonzero(np.all((lo - h <= x0) & (x0 <= hi + h), axis=1))[0]
                if near.size == 0:
                    continue
                g = np.asarray(gamma[k], dtype=np.float64)
                for sid in near:
                    b = A.block(k, sid)
                    P = A.P[b]
                    d_excl = np.where(A.i1[b] != row, A.d1[b], A.d2[b])
                    n_excl = np.where(A.i1[b] != row, A.i1[b], A.i2[b])
                    j0 = int(np.argmax(A.d1[b]))
                    n0 = int(A.i1[b][j0])
                    for sgn in (+1.0, -1.0):
                        xp = x0.copy()
                        xp[col] += sgn * h
                        dm = np.linalg.norm(P - xp, axis=1)
                        moved_wins = (dm < d_excl) | ((dm == d_excl) & (row < n_excl))
                        dnew = np.where(moved_wins, dm, d_excl)
                        nnew = np.where(moved_wins, row, n_excl)
                        j = int(np.argmax(dnew))
                        if sgn > 0:
                            plus += g[sid] * dnew[j]
                        else:
                            minus += g[sid] * dnew[j]
                        changed |= (j != j0) or (int(nnew[j]) != n0)
                    # simplices whose values are unchanged contribute equally to both sides
        fd[t] = (plus - minus) / (2.0 * h)
        kink[t] = changed
    return fd, kink, cache
