"""Flood values for arbitrary finite point sets P_sigma, in FP64 (§4.1, Theorem 2, Lemma 4).

Test infrastructure: only tests, the smoke check and the benchmark's CPU
baseline may import this module.

§4.1 replaces each conv(sigma) by a finite P_sigma ⊂ conv(sigma) and defines

    Flood_r(X, L, P) = { sigma in Del(L) : P_tau ⊂ X_r for every face tau of sigma },

so a simplex enters at the smallest r at which the points of all its faces
(itself included) are within r of X:

    f_P(sigma) = max over faces tau ⊆ sigma of  max_{p in P_tau} min_{x in X} |p - x|.

The paper names random draws as one choice of P (§4.1; Lemma 4 bounds the
Hausdorff distance of a uniform sample). Here every simplex of dimension
k >= 1 carries its own set, given as barycentric coordinates

    weights[k][row, s] = (lambda_0, ..., lambda_k),   lambda_j >= 0, sum = 1,

and the point is p = sum_j lambda_j v_j with v_j the rows of L named by the
simplex's ascending vertex ids. lambda_0 is taken as 1 - sum_{j>=1} lambda_j,
which equals the stored value whenever the weights sum to one; it is the
coefficient of v_0 in p = v_0 + sum_{j>=1} lambda_j (v_j - v_0). A vertex's
set is the vertex itself (P_v = {v}; f(v) = d(v, X), 0 when L ⊂ X).

This module enumerates the faces of each simplex explicitly (every non-empty
subset of its vertices, looked up in the simplex lists) rather than using any
recursion over facets, and takes nearest distances by brute force or with the
exact k-d tree of flood.py.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import combinations

import numpy as np

from .flood import KDIndex

__all__ = ["RandomFloodResult", "random_points", "own_maxima", "flood_values_random",
           "analytic_gradient_random", "total_random"]


@dataclass
class RandomFloodResult:
    values: list        # k -> float64 (n_k,): f_P(sigma)
    src: list           # k -> int64 (n_k, 3): (dim, row, sample) of the attaining point
    argmin_point: list  # k -> int64 (n_k,): nearest row of X to the attaining point
    own: list           # k -> float64 (n_k,): max over the simplex's own set (-inf if empty)


def lambdas(weights_row: np.ndarray) -> np.ndarray:
    """FP64 barycentric coordinates with lambda_0 = 1 - sum_{j>=1} lambda_j."""
    lam = np.asarray(weights_row, dtype=np.float64).copy()
    lam[..., 0] = 1.0 - lam[..., 1:].sum(axis=-1)
    return lam


def random_points(V: np.ndarray, weights_row: np.ndarray) -> np.ndarray:
    """p = sum_j lambda_j v_j for one simplex: V (k+1, 3), weights (S, k+1) -> (S, 3)."""
    return lambdas(weights_row) @ np.asarray(V, dtype=np.float64)


def own_maxima(X, L, simplices, weights, index: KDIndex):
    """Per simplex: max over its own set of the nearest distance, the sample
    attaining it (lowest index on ties) and that sample's nearest row of X."""
    L64 = np.asarray(L, dtype=np.float64)
    own, arg, near = [], [], []
    d0, i0 = index.query(L64)
    own.append(np.asarray(d0, dtype=np.float64).reshape(-1))
    arg.append(np.zeros(L64.shape[0], dtype=np.int64))
    near.append(np.asarray(i0, dtype=np.int64).reshape(-1))
    for k in range(1, len(simplices)):
        S = np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1)
        W = np.asarray(weights[k], dtype=np.float64).reshape(S.shape[0], -1, k + 1)
        n, ns = S.shape[0], W.shape[1]
        val = np.full(n, -np.inf)
        am = np.full(n, -1, dtype=np.int64)
        an = np.full(n, -1, dtype=np.int64)
        if n and ns:
            P = np.einsum("nsj,njd->nsd", lambdas(W), L64[S])         # (n, S, 3)
            d, i = index.query(P.reshape(-1, 3))
            d = d.reshape(n, ns)
            i = i.reshape(n, ns)
            am = np.argmax(d, axis=1)                                  # first maximum: lowest sample
            val = d[np.arange(n), am]
            an = i[np.arange(n), am]
        own.append(val)
        arg.append(am)
        near.append(an)
    return own, arg, near


def flood_values_random(X, L, simplices, weights, method: str = "brute",
                        index: KDIndex | None = None) -> RandomFloodResult:
    """f_P(sigma) = max over all faces tau ⊆ sigma of max_{p in P_tau} d(p, X).

    simplices: k -> (n_k, k+1) ascending rows of L (k = 0 may be None: the
    vertices are the rows of L). weights: k -> (n_k, S_k, k+1) for k >= 1
    (weights[0] is ignored). Every face of a listed simplex must itself be
    listed. Ties between attaining points go to the lowest (dim, row, sample).
    """
    if index is None:
        index = KDIndex(X, method)
    n_l = np.asarray(L).shape[0]
    own, arg, near = own_maxima(X, L, simplices, weights, index)
    lookup = [None] + [{tuple(int(v) for v in row): r
                        for r, row in enumerate(np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1))}
                       for k in range(1, len(simplices))]
    values, src, amin = [], [], []
    for k in range(len(simplices)):
        S = (np.arange(n_l, dtype=np.int64).reshape(-1, 1) if k == 0
             else np.asarray(simplices[k], dtype=np.int64).reshape(-1, k + 1))
        val = np.empty(S.shape[0])
        sr = np.empty((S.shape[0], 3), dtype=np.int64)
        an = np.empty(S.shape[0], dtype=np.int64)
        for r, verts in enumerate(S):
            best = None                              # (-value, dim, row, sample)
            for size in range(1, k + 2):
                for face in combinations(tuple(int(v) for v in verts), size):
                    dim = size - 1
                    row = face[0] if dim == 0 else lookup[dim].get(face)
                    if row is None:
                        raise ValueError(f"face {face} of simplex {tuple(verts)} is not listed")
                    if not np.isfinite(own[dim][row]):
                        continue                     # an empty set adds nothing
                    cand = (-own[dim][row], dim, row, int(arg[dim][row]))
                    if best is None or cand < best:
                        best = cand
            val[r] = -best[0]
            sr[r] = best[1:]
            an[r] = near[best[1]][best[2]]
        values.append(val)
        src.append(sr)
        amin.append(an)
    return RandomFloodResult(values, src, amin, own)


def total_random(result: RandomFloodResult, gamma) -> float:
    """F = sum over k >= 0 of sum_sigma gamma_sigma f_P(sigma) (vertices included)."""
    return float(sum(np.dot(np.asarray(gamma[k], np.float64), result.values[k])
                     for k in range(len(result.values))))


def analytic_gradient_random(X, L, simplices, weights, gamma, result: RandomFloodResult):
    """(dX (N,3), dL (n_L,3)) of F = sum gamma f_P in FP64.

    On a smooth piece f_P(sigma) = |p* - x*| with p* = sum_j lambda_j v_j the
    attaining point of the attaining face tau and x* its nearest point of X:
    d f / d x* = (x* - p*) / f and d f / d v_j = lambda_j (p* - x*) / f over
    tau's vertices (lambda_0 = 1 - sum_{j>=1} lambda_j); a vertex tau is the
    point itself (lambda = 1); f = 0 gives zero.
    """
    X64 = np.asarray(X, dtype=np.float64)
    L64 = np.asarray(L, dtype=np.float64)
    dX = np.zeros_like(X64)
    dL = np.zeros_like(L64)
    for k in range(len(result.values)):
        g = np.asarray(gamma[k], dtype=np.float64)
        for r in range(result.values[k].shape[0]):
            dim, row, s = (int(v) for v in result.src[k][r])
            if dim == 0:                             # a vertex attains: p* = v
                verts = np.array([row])
                lam = np.ones(1)
            else:
                verts = np.asarray(simplices[dim], dtype=np.int64).reshape(-1, dim + 1)[row]
                lam = lambdas(np.asarray(weights[dim], dtype=np.float64).reshape(
                    np.asarray(simplices[dim]).reshape(-1, dim + 1).shape[0], -1, dim + 1)[row, s])
            p = lam @ L64[verts]
            xi = int(result.argmin_point[k][r])
            f = float(np.linalg.norm(p - X64[xi]))
            if not f > 0.0:
                continue
            u = (p - X64[xi]) / f
            dX[xi] -= g[r] * u
            for j in range(dim + 1):
                dL[verts[j]] += g[r] * lam[j] * u
    return dX, dL
