"""Farthest point sampling (FPS) oracle.

The paper selects landmarks L ⊂ X by farthest point sampling, the greedy
k-centre heuristic whose covering radius is within a factor 2 of optimal
(§3.2, after Corollary 1; used in §5.1, §5.3 and App. B.3). It does not state
the start point, the tie rule or the precision. The reading adopted here:

  * l_0 = X[start];
  * d_i = +inf, then for j = 1 .. n-1:  d_i <- min(d_i, kappa(x_i, l_{j-1})),
    l_j = argmax_i d_i with ties broken towards the LOWEST index;
  * kappa is the squared Euclidean distance evaluated in IEEE binary32 with
    every operation rounded separately (no fused multiply-add):
        dx = fl32(x.x - l.x), ...;  kappa = fl32(fl32(fl32(dx*dx) + fl32(dy*dy)) + fl32(dz*dz)),
    and in d coordinates the squares summed left to right in the same way
    (the ambient dimension is free in §3; Fig. 4c varies it).

kappa decides an integer (the argmax), so it is evaluated in binary32 on both
sides. numpy's float32 element-wise arithmetic is IEEE binary32 with one
rounding per operation, which is the same value as computing each operation
in FP64 and rounding it to binary32 (53 >= 2*24 + 2, so the double rounding is
innocuous for +, -, *); tests pin that equivalence.
"""
from __future__ import annotations

import numpy as np

__all__ = ["fps", "fps_key", "DegenerateFPS"]


class DegenerateFPS(ValueError):
    """FPS ran out of distinct points (the maximum key became 0 before n picks)."""


def fps_key(X: np.ndarray, l: np.ndarray) -> np.ndarray:
    """kappa(x_i, l) for all rows x_i of float32 X (n, d), in binary32 without contraction."""
    X = np.asarray(X, dtype=np.float32)
    l = np.asarray(l, dtype=np.float32)
    d0 = X[:, 0] - l[0]
    acc = d0 * d0
    for c in range(1, X.shape[1]):
        dc = X[:, c] - l[c]
        acc = acc + dc * dc
    return acc


def fps(X: np.ndarray, n_landmarks: int, start: int = 0):
    """Return (idx int64[n], key float32[n]); key[j] = d_{idx[j]} when it was picked.

    key[0] is +inf (the start point is given, not picked). Raises DegenerateFPS
    when fewer than n distinct points exist.
    """
    X = np.ascontiguousarray(X, dtype=np.float32)
    N = X.shape[0]
    if not (1 <= n_landmarks <= N):
        raise ValueError("need 1 <= n_landmarks <= N")
    if not (0 <= start < N):
        raise ValueError("start out of range")
    d = np.full(N, np.inf, dtype=np.float32)
    idx = np.empty(n_landmarks, dtype=np.int64)
    key = np.empty(n_landmarks, dtype=np.float32)
    idx[0], key[0] = start, np.inf
    cur = start
    for j in range(1, n_landmarks):
        np.minimum(d, fps_key(X, X[cur]), out=d)
        cur = int(np.argmax(d))          # first maximum = lowest index among ties
        if not d[cur] > 0:
            raise DegenerateFPS(f"only {j} distinct points")
        idx[j], key[j] = cur, d[cur]
    return idx, key
