"""Pins of the oracle in ambient dimensions 4 and 5 (§3 leaves d free; §5.3, Fig. 4c varies it).

Checked against what the mathematics fixes, not against the oracle itself:
  * FPS on the vertices of the unit 4-cube: the farthest-point order and its
    keys follow from the Hamming weights (every squared distance is an integer).
  * FPS with d-coordinate keys on a cloud whose extra coordinates are 0 picks
    exactly what 3-coordinate FPS picks on the first three (adding an exact 0).
  * The flood value of a regular d-simplex over its own vertices is its
    circumradius a*sqrt(d/(2(d+1))) when (d+1) | m (the barycentre is a
    grid point and the farthest point of the simplex from its vertices).
  * An edge between two points of X alone: half its length for even m.
  * Flood values are invariant under a rotation of X and L (every coordinate
    enters the distance; dropping one breaks this).
  * The k-d tree agrees with brute force in 5-D.
  * The host Delaunay complex of 5-D landmarks is closed under faces with
    consistent facet incidence (every facet row is the simplex minus one vertex).
"""
import numpy as np
import pytest

import oracle
from paper_2509_22432_b300 import complex_from_simplices, data, delaunay_complex


def _regular_simplex(d: int, a: float = 1.0) -> np.ndarray:
    """d+1 vertices of a regular d-simplex with edge a, in R^d."""
    E = np.eye(d + 1)                                  # regular simplex in the plane sum = 1 of R^{d+1}
    E = E - E.mean(axis=0)
    # orthonormal basis of the plane
    Q, _ = np.linalg.qr(E.T)
    V = E @ Q[:, :d]
    V *= a / np.linalg.norm(V[0] - V[1])
    return V


def test_fps_on_the_4_cube_follows_hamming_weights():
    X = np.array([[(i >> b) & 1 for b in (3, 2, 1, 0)] for i in range(16)], dtype=np.float32)
    idx, key = oracle.fps(X, 5, 0)
    # from 0000 the farthest vertex is 1111 (squared distance 4); after both, a vertex of
    # Hamming weight w is at min(w, 4 - w): the weight-2 vertices tie at 2, lowest index 0011
    assert idx[0] == 0 and idx[1] == 15 and key[1] == 4.0
    assert idx[2] == 3 and key[2] == 2.0
    # each later pick is the lowest-index maximiser of the distance to the picks so far
    for j in range(3, 5):
        picked = X[idx[:j]]
        d2 = ((X[:, None, :] - picked[None]) ** 2).sum(-1).min(1)
        assert key[j] == d2.max() and idx[j] == int(np.argmax(d2))


@pytest.mark.parametrize("d", [4, 5])
def test_fps_extra_zero_coordinates_change_nothing(d):
    X3 = data.sphere_cloud(3000, seed=71)
    Xd = np.zeros((X3.shape[0], d), np.float32)
    Xd[:, :3] = X3
    a = oracle.fps(X3, 40, 5)
    b = oracle.fps(Xd, 40, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


def test_fps_uses_every_coordinate():
    rng = np.random.default_rng(72)
    X = rng.standard_normal((2000, 5)).astype(np.float32)
    full = oracle.fps(X, 30, 0)[0]
    X4 = X.copy()
    X4[:, 4] = 0
    assert not np.array_equal(full, oracle.fps(X4, 30, 0)[0])


@pytest.mark.parametrize("d,m", [(4, 5), (4, 10), (5, 6), (5, 12)])
def test_regular_simplex_value_is_its_circumradius(d, m):
    V = _regular_simplex(d, a=1.5)
    cx = complex_from_simplices([np.arange(d + 1)[None]], d + 1)
    r = oracle.flood_values(V.astype(np.float32), V.astype(np.float32), cx.simplices, m)
    R = 1.5 * np.sqrt(d / (2.0 * (d + 1)))
    Vf = V.astype(np.float32).astype(np.float64)
    c = Vf.mean(axis=0)
    Rf = np.linalg.norm(Vf - c, axis=1).min()           # float32 rounding of the vertices
    assert abs(r.values[d][0] - Rf) < 1e-12 and abs(Rf - R) < 1e-6
    # an edge alone: half its length (m even)
    if m % 2 == 0:
        e = np.linalg.norm(Vf[0] - Vf[1])
        assert np.isclose(r.values[1], e / 2, atol=1e-12).all()


def test_values_are_rotation_invariant_in_5d():
    rng = np.random.default_rng(73)
    X = rng.uniform(0, 1, (3000, 5))
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    idx = rng.choice(3000, 14, replace=False)
    L = X[idx]
    cx = delaunay_complex(L.astype(np.float32))
    a = oracle.flood_values(X, L, cx.simplices, 6, method="kdtree")
    b = oracle.flood_values(X @ Q, L @ Q, cx.simplices, 6, method="kdtree")
    for k in range(6):
        assert np.allclose(a.values[k], b.values[k], rtol=1e-12, atol=1e-12), k


def test_kdtree_equals_brute_force_in_5d():
    rng = np.random.default_rng(74)
    X = rng.uniform(-1, 1, (4000, 5)).astype(np.float32)
    Q = rng.uniform(-1.2, 1.2, (500, 5))
    db, ib = oracle.flood.KDIndex(X, "brute").query(Q)
    dk, ik = oracle.flood.KDIndex(X, "kdtree").query(Q)
    assert np.allclose(db, dk, rtol=0, atol=1e-12)
    assert np.array_equal(ib, ik)


@pytest.mark.parametrize("d", [4, 5])
def test_delaunay_complex_in_d_dimensions(d):
    X = data.swisscheese_cloud(3000, seed=75, dim=d)
    L = X[oracle.fps(X, 60, 0)[0]]
    cx = delaunay_complex(L)
    assert cx.top_dim == d and cx.counts[d] > 0
    for k in range(2, d + 1):
        s, f = cx.simplices[k], cx.facets[k]
        for j in range(k + 1):
            assert np.array_equal(cx.simplices[k - 1][f[:, j]], np.delete(s, j, axis=1))
    # Euler characteristic of a triangulated d-ball is 1
    assert sum((-1) ** k * n for k, n in enumerate(cx.counts)) == 1
    assert data.swisscheese_cloud(3000, seed=75, dim=d).shape == (3000, d)
