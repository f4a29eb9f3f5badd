"""Pins of the random-P_sigma oracle (§4.1 with given point sets, Lemma 4) against
what the mathematics fixes (CPU only).

- Special case that reduces to an already pinned routine: when every simplex's
  set is its interior barycentric grid, the face-enumerated maximum is the
  full-grid value of Lemma 1 (the grid oracle).
- Closed forms: centroid / midpoint sets on the equilateral triangle and the
  regular tetrahedron (circumradius), an empty own set (the faces decide).
- Exact inequalities from d(., X) being 1-Lipschitz: the grid value of Lemma 1
  bounds f_P from above (+ the Lemma 1 covering radius) and from below (- the
  largest distance from a grid point to the nearest point of the sets).
- Invariants: P ⊂ P' gives f_P <= f_P'; face <= coface; brute force = k-d tree.
- The analytic subgradient against central differences of the oracle's own F.
"""
import math
from itertools import combinations

import numpy as np
import pytest

import oracle
from oracle.flood import KDIndex
from paper_2509_22432_b300 import data
from paper_2509_22432_b300.complex import complex_from_simplices, delaunay_complex


def _cx(simplices, n_vertices):
    return complex_from_simplices([np.asarray(simplices)], n_vertices).simplices


def _grid_weights(simplices, m):
    """Every simplex of dimension k >= 1 gets the interior compositions c/m."""
    w = [None]
    for k in range(1, len(simplices)):
        lam = oracle.interior_compositions(m, k).astype(np.float64) / m
        w.append(np.broadcast_to(lam, (np.asarray(simplices[k]).shape[0],) + lam.shape).copy())
    return w


def _cloud(n, n_l, seed):
    X = data.torus_cloud(n, seed=seed)
    idx, _ = oracle.fps(X, n_l)
    L = X[idx]
    return X, L, delaunay_complex(L)


def test_interior_grid_sets_reproduce_the_full_grid_value():
    """P_tau = interior grid of tau for every face: the union over faces is the full grid of Lemma 1."""
    X, L, cx = _cloud(3000, 30, seed=91)
    for m in (3, 5, 6):
        grid = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
        rnd = oracle.flood_values_random(X, L, cx.simplices, _grid_weights(cx.simplices, m), method="kdtree")
        for k in range(4):
            assert np.allclose(rnd.values[k], grid.values[k], rtol=0, atol=1e-12), (m, k)


def _equilateral():
    a = 1.0
    V = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]], dtype=np.float64)
    V += np.array([0.75, -0.5, 0.25])      # off the origin, so that lambda_0 matters
    return a, V, _cx([[0, 1, 2]], 3)


def test_centroid_and_midpoint_sets_on_the_equilateral_triangle():
    a, V, S = _equilateral()
    w = [None, np.full((3, 1, 2), 0.5), np.full((1, 1, 3), 1.0 / 3.0)]
    r = oracle.flood_values_random(V, V, S, w)
    assert np.allclose(r.values[1], a / 2, rtol=0, atol=1e-12)
    assert abs(r.values[2][0] - a / math.sqrt(3)) <= 1e-12
    assert tuple(r.src[2][0]) == (2, 0, 0)


def test_off_centre_point_and_lambda0_is_implied():
    """lambda = (1/2, 1/4, 1/4): p = v0/2 + (v1 + v2)/4; the stored lambda_0 is not read."""
    a, V, S = _equilateral()
    p = 0.5 * V[0] + 0.25 * V[1] + 0.25 * V[2]
    d = min(np.linalg.norm(p - v) for v in V)
    for lam0 in (0.5, 0.0, 7.0):
        w = [None, np.zeros((3, 0, 2)), np.array([[[lam0, 0.25, 0.25]]])]
        r = oracle.flood_values_random(V, V, S, w)
        assert abs(r.values[2][0] - d) <= 1e-12
        assert np.all(r.values[1] == 0.0)          # empty edge sets: only the vertices (value 0)


def test_regular_tetrahedron_with_centroid_sets():
    a = 2 * math.sqrt(2)
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    S = _cx([[0, 1, 2, 3]], 4)
    w = [None, np.full((6, 1, 2), 0.5), np.full((4, 1, 3), 1.0 / 3.0), np.full((1, 1, 4), 0.25)]
    r = oracle.flood_values_random(V, V, S, w)
    assert abs(r.values[3][0] - a * math.sqrt(6) / 4) <= 1e-12
    # without its own point the tetrahedron takes its triangles' centroid value a / sqrt(3)
    w[3] = np.zeros((1, 0, 4))
    r = oracle.flood_values_random(V, V, S, w)
    assert abs(r.values[3][0] - a / math.sqrt(3)) <= 1e-12
    assert r.src[3][0][0] == 2


def _lemma1_radius(V):
    V = np.asarray(V, np.float64)
    return math.sqrt(sum(np.sum((V[i] - V[j]) ** 2) for i, j in combinations(range(len(V)), 2)))


@pytest.mark.parametrize("seed", [101, 102])
def test_grid_value_brackets_the_random_value(seed):
    """1-Lipschitz d(., X): f_grid - D <= f_P <= f_grid + radius(Lemma 1) / m, with D the
    largest distance from a full-grid point of sigma to the nearest point of the sets of
    sigma's faces (vertices included)."""
    X, L, cx = _cloud(4000, 30, seed=seed)
    L64 = L.astype(np.float64)
    m = 6
    w = [None] + [data.random_barycentric(cx.counts[k], 12, k, seed=seed) for k in range(1, 4)]
    rnd = oracle.flood_values_random(X, L, cx.simplices, w, method="kdtree")
    grid = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
    lookup = [None] + [{tuple(r): i for i, r in enumerate(cx.simplices[k].tolist())} for k in range(1, 4)]
    for k in range(1, 4):
        full = oracle.compositions(m, k) / m
        for r, verts in enumerate(cx.simplices[k]):
            V = L64[verts]
            assert rnd.values[k][r] <= grid.values[k][r] + _lemma1_radius(V) / m + 1e-12
            pts = [L64[v] for v in verts]
            for size in range(2, k + 2):
                for face in combinations(verts.tolist(), size):
                    lam = w[size - 1][lookup[size - 1][face]].astype(np.float64)
                    lam = lam.copy()
                    lam[:, 0] = 1.0 - lam[:, 1:].sum(axis=1)
                    pts.extend(lam @ L64[list(face)])
            P = np.array(pts)
            Q = full @ V
            D = np.sqrt(((Q[:, None, :] - P[None, :, :]) ** 2).sum(axis=2)).min(axis=1).max()
            assert rnd.values[k][r] >= grid.values[k][r] - D - 1e-12


def test_more_points_never_lower_the_value_and_faces_stay_below():
    X, L, cx = _cloud(4000, 40, seed=111)
    w = [None] + [data.random_barycentric(cx.counts[k], 16, k, seed=112) for k in range(1, 4)]
    half = [None] + [wk[:, :8] for wk in w[1:]]
    ind = KDIndex(X, "kdtree")
    big = oracle.flood_values_random(X, L, cx.simplices, w, index=ind)
    small = oracle.flood_values_random(X, L, cx.simplices, half, index=ind)
    for k in range(1, 4):
        assert np.all(small.values[k] <= big.values[k])
        fac = big.values[k - 1][cx.facets[k]] if k >= 2 else big.values[0][cx.simplices[1]]
        assert np.all(fac.max(axis=1) <= big.values[k])


def test_brute_force_equals_kdtree():
    X, L, cx = _cloud(3000, 24, seed=121)
    w = [None] + [data.random_barycentric(cx.counts[k], 10, k, seed=122) for k in range(1, 4)]
    a = oracle.flood_values_random(X, L, cx.simplices, w, method="brute")
    b = oracle.flood_values_random(X, L, cx.simplices, w, method="kdtree")
    for k in range(4):
        assert np.allclose(a.values[k], b.values[k], rtol=0, atol=1e-12)


def test_random_gradient_matches_central_differences():
    X = data.jitter(data.torus_cloud(500, seed=131), amp=1e-6, seed=132)
    idx, _ = oracle.fps(X, 14)
    L = X[idx].astype(np.float64)
    X = X.astype(np.float64)
    cx = delaunay_complex(L)
    w = [None] + [data.random_barycentric(cx.counts[k], 6, k, seed=133) for k in range(1, 4)]
    gamma = data.upstream_gradients(cx.counts, seed=134)
    base = oracle.flood_values_random(X, L, cx.simplices, w)
    dX, dL = oracle.analytic_gradient_random(X, L, cx.simplices, w, gamma, base)
    rng = np.random.default_rng(5)
    nz = np.argwhere(np.abs(dX) > 0)
    probes = [("X", int(a), int(b)) for a, b in nz[rng.choice(len(nz), min(25, len(nz)), replace=False)]]
    nzl = np.argwhere(np.abs(dL) > 0)
    probes += [("L", int(a), int(b)) for a, b in nzl[rng.choice(len(nzl), min(15, len(nzl)), replace=False)]]
    probes += [("X", int(a), 2) for a in rng.choice(X.shape[0], 5)]
    h = 1e-6
    n_ok = 0
    for which, row, col in probes:
        F, same = [], True
        for sgn in (1.0, -1.0):
            Xp, Lp = X.copy(), L.copy()
            (Xp if which == "X" else Lp)[row, col] += sgn * h
            r = oracle.flood_values_random(Xp, Lp, cx.simplices, w)
            F.append(oracle.total_random(r, gamma))
            for k in range(1, 4):
                same &= np.array_equal(r.src[k], base.src[k]) and np.array_equal(r.argmin_point[k],
                                                                                  base.argmin_point[k])
        if not same:
            continue                                      # a kink inside +-h: one-sided, not compared
        fd = (F[0] - F[1]) / (2 * h)
        an = dX[row, col] if which == "X" else dL[row, col]
        assert abs(fd - an) <= 1e-3 * abs(an) + 1e-5, (which, row, col, fd, an)
        n_ok += 1
    assert n_ok >= 30


def test_random_sets_with_landmarks_off_X():
    """Vertices off X: f(v) = d(v, X) > 0 enters every coface; gradient still matches FD."""
    X = data.jitter(data.torus_cloud(500, seed=161), amp=1e-6, seed=162).astype(np.float64)
    idx, _ = oracle.fps(X, 12)
    rng = np.random.default_rng(163)
    L = X[idx] + rng.uniform(-0.05, 0.05, (12, 3))
    cx = delaunay_complex(L)
    w = [None] + [data.random_barycentric(cx.counts[k], 4, k, seed=164) for k in range(1, 4)]
    gamma = data.upstream_gradients(cx.counts, seed=165)
    base = oracle.flood_values_random(X, L, cx.simplices, w)
    d, _ = KDIndex(X, "brute").query(L)
    assert np.allclose(base.values[0], d, rtol=0, atol=1e-12) and np.all(d > 0)
    for k in range(1, 4):
        verts = np.asarray(cx.simplices[k])
        assert np.all(base.values[k] >= d[verts].max(axis=1))
    dX, dL = oracle.analytic_gradient_random(X, L, cx.simplices, w, gamma, base)
    h, n_ok = 1e-6, 0
    for row in range(12):
        for col in range(3):
            F, same = [], True
            for sgn in (1.0, -1.0):
                Lp = L.copy()
                Lp[row, col] += sgn * h
                r = oracle.flood_values_random(X, Lp, cx.simplices, w)
                F.append(oracle.total_random(r, gamma))
                same &= all(np.array_equal(r.src[k], base.src[k]) and
                            np.array_equal(r.argmin_point[k], base.argmin_point[k]) for k in range(4))
            if same:
                assert abs((F[0] - F[1]) / (2 * h) - dL[row, col]) <= 1e-3 * abs(dL[row, col]) + 1e-5
                n_ok += 1
    assert n_ok >= 25
