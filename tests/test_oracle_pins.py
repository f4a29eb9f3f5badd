"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: closed forms
(edge, equilateral triangle, regular tetrahedron, circle example of App. C.3),
inequalities the paper proves (Lemma 1 covering bound, Lemma 2 masking,
Theorem 1 stability, the circumradius bound of the Alpha/Flood lemma in
App. C), invariants (face <= coface, FPS packing/covering, exact scaling),
library routines on special cases (brute force vs k-d tree), brute force on
tiny inputs (optimal k-centre radius), and Betti numbers from independent
rank computations for the persistence reduction.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle.fps import DegenerateFPS
from oracle.flood import ritter_ball, KDIndex
from paper_2509_22432_b300.complex import complex_from_simplices, delaunay_complex
from paper_2509_22432_b300 import data


# ----------------------------------------------------------------------------- FPS

def test_fps_key_matches_fp64_rounded_per_operation():
    """numpy binary32 arithmetic == FP64 evaluation rounded to binary32 after each op."""
    rng = np.random.default_rng(0)
    X = (rng.standard_normal((20000, 3)) * rng.choice([1e-3, 1.0, 37.0], (20000, 1))).astype(np.float32)
    l = X[123]
    r32 = lambda a: np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)
    X64, l64 = X.astype(np.float64), l.astype(np.float64)
    dx, dy, dz = (r32(X64[:, c] - l64[c]) for c in range(3))
    ref = r32(r32(r32(dx * dx) + r32(dy * dy)) + r32(dz * dz))
    got = oracle.fps_key(X, l).astype(np.float64)
    assert np.array_equal(got, ref)


def _circle(n, z=0.0):
    t = 2 * np.pi * np.arange(n) / n
    return np.stack([np.cos(t), np.sin(t), np.full(n, z)], axis=1).astype(np.float32)


def test_fps_circle_stages():
    """App. C.3: stage k of FPS on the circle picks exactly the angles 2*pi*j/2^k."""
    n = 1024
    X = _circle(n)
    idx, key = oracle.fps(X, n_landmarks=256, start=0)
    for k in range(1, 9):
        got = set(idx[: 2 ** k].tolist())
        want = set(range(0, n, n // 2 ** k))
        assert got == want, k


@pytest.mark.parametrize("n_l", [3, 5, 12, 13, 20, 33])
def test_fps_circle_short_arc_count(n_l):
    """App. C.3: 2(|L| - 2^floor(log2 |L|)) short arcs of length pi / 2^floor(log2 |L|)."""
    n = 4096
    idx, _ = oracle.fps(_circle(n), n_landmarks=n_l, start=0)
    s = np.sort(idx)
    arcs = np.diff(np.concatenate([s, [s[0] + n]]))
    a = 2 ** int(math.floor(math.log2(n_l)))
    short = n // (2 * a)
    assert np.sum(arcs == short) == 2 * (n_l - a)
    assert np.sum(arcs == 2 * short) == n_l - 2 * (n_l - a)


def test_fps_two_approximation_of_k_centre():
    """§3.2: FPS covering radius <= 2 x the optimal k-centre radius (brute force, tiny sets)."""
    rng = np.random.default_rng(1)
    for trial in range(20):
        X = rng.standard_normal((9, 3)).astype(np.float32)
        X64 = X.astype(np.float64)
        D = np.linalg.norm(X64[:, None] - X64[None], axis=2)
        k = 3
        opt = min(D[:, list(c)].min(axis=1).max() for c in itertools.combinations(range(9), k))
        for start in range(9):
            idx, _ = oracle.fps(X, k, start=start)
            cover = D[:, idx].min(axis=1).max()
            assert cover <= 2 * opt + 1e-12


def test_fps_covering_and_packing():
    """key[j+1] is the squared covering radius of the first j+1 landmarks; landmarks are packed."""
    X = data.sphere_cloud(3000, seed=11)
    idx, key = oracle.fps(X, 60, start=0)
    X64 = X.astype(np.float64)
    assert np.all(np.diff(key[1:]) <= 0)
    for j in [1, 5, 17, 40, 58]:
        Lj = X64[idx[: j + 1]]
        cover2 = (np.linalg.norm(X64[:, None] - Lj[None], axis=2).min(axis=1) ** 2).max()
        assert abs(cover2 - key[j + 1]) <= 1e-6 * key[j + 1]
    Lall = X64[idx]
    D = np.linalg.norm(Lall[:, None] - Lall[None], axis=2) ** 2
    D[np.diag_indices_from(D)] = np.inf
    assert D.min() >= key[-1] * (1 - 1e-6)


def test_fps_scaling_by_two_is_exact():
    X = data.sphere_cloud(2000, seed=12)
    i1, k1 = oracle.fps(X, 50, 7)
    i2, k2 = oracle.fps(2 * X, 50, 7)
    assert np.array_equal(i1, i2)
    assert np.array_equal(4 * k1[1:], k2[1:])


def test_fps_ties_go_to_lowest_index_and_degenerate_raises():
    X = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 0, 0]], dtype=np.float32)
    idx, key = oracle.fps(X, 3, 0)
    assert idx.tolist() == [0, 1, 2]
    with pytest.raises(DegenerateFPS):
        oracle.fps(X, 4, 0)


# ----------------------------------------------------------------------------- samples

@pytest.mark.parametrize("m", [1, 2, 6, 8, 10, 12, 19])
def test_grid_counts(m):
    for k in range(4):
        assert oracle.compositions(m, k).shape[0] == math.comb(m + k, k)
        assert oracle.interior_compositions(m, k).shape[0] == (math.comb(m - 1, k) if k <= m - 1 else 0)
    if m == 19:   # "20 points per edge" -> 210 per triangle, 1540 per tetrahedron (§5.3)
        assert oracle.compositions(19, 2).shape[0] == 210
        assert oracle.compositions(19, 3).shape[0] == 1540


@pytest.mark.parametrize("m,k", [(6, 2), (12, 3), (5, 1), (8, 3)])
def test_grid_is_interior_plus_facet_grids(m, k):
    """P_tau ⊂ P_sigma for faces (App. A.1): the full grid = interior ∪ the facets' full grids."""
    full = {tuple(c) for c in oracle.compositions(m, k)}
    interior = {tuple(c) for c in oracle.interior_compositions(m, k)}
    faces = set()
    for j in range(k + 1):
        for c in oracle.compositions(m, k - 1):
            faces.add(tuple(np.insert(c, j, 0)))
    assert interior.isdisjoint(faces)
    assert full == interior | faces
    comps = oracle.compositions(m, k)
    assert all(tuple(a) < tuple(b) for a, b in zip(comps[:-1], comps[1:]))   # lexicographic


@pytest.mark.parametrize("k,m", [(1, 3), (2, 5), (3, 4), (3, 7)])
def test_lemma1_covering_bound(k, m):
    """Lemma 1: every point of conv(sigma) is within (1/m) sqrt(sum_{i<j}|vi-vj|^2) of P_sigma."""
    rng = np.random.default_rng(k * 10 + m)
    V = rng.standard_normal((k + 1, 3)) + np.array([7.0, -3.0, 5.0])   # away from the origin
    P = oracle.sample_points(V, oracle.compositions(m, k), m)
    bound = math.sqrt(sum(np.sum((V[i] - V[j]) ** 2) for i in range(k + 1) for j in range(i))) / m
    lam = rng.dirichlet(np.ones(k + 1), 4000)
    lam = np.concatenate([lam, np.eye(k + 1)])
    Q = lam @ V
    d = np.linalg.norm(Q[:, None] - P[None], axis=2).min(axis=1)
    assert d.max() <= bound + 1e-12


# ----------------------------------------------------------------------------- flood values

def _cx(simplices, n_vertices):
    return complex_from_simplices([np.asarray(simplices)], n_vertices).simplices


def test_vertex_values_are_zero_when_L_subset_X():
    X = data.sphere_cloud(500, seed=3)
    idx, _ = oracle.fps(X, 10)
    r = oracle.flood_values(X, X[idx], [np.arange(10)[:, None]], m=4)
    assert np.all(r.values[0] == 0.0)


@pytest.mark.parametrize("m", [2, 4, 6, 12])
def test_edge_between_its_two_points_is_half_length(m):
    V = np.array([[0.1, -0.3, 0.2], [1.3, 0.4, -0.5]], dtype=np.float32)
    r = oracle.flood_values(V, V, [np.zeros((0, 1), np.int64), np.array([[0, 1]])], m=m)
    ell = np.linalg.norm(V[0].astype(np.float64) - V[1])
    assert abs(r.values[1][0] - ell / 2) <= 1e-12


@pytest.mark.parametrize("m", [3, 6, 12])
def test_equilateral_triangle_reaches_circumradius(m):
    """App. C (Flood <= Alpha lemma): f = circumradius a/sqrt(3) when the centroid is a sample."""
    a = 1.0
    V = np.array([[0, 0, 0], [a, 0, 0], [a / 2, a * math.sqrt(3) / 2, 0]], dtype=np.float64)
    S = _cx([[0, 1, 2]], 3)
    r = oracle.flood_values(V, V, S, m=m)
    assert abs(r.values[2][0] - a / math.sqrt(3)) <= 1e-9


@pytest.mark.parametrize("m", [4, 8, 12])
def test_regular_tetrahedron_reaches_circumradius(m):
    a = 2 * math.sqrt(2)
    V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    S = _cx([[0, 1, 2, 3]], 4)
    r = oracle.flood_values(V, V, S, m=m)
    assert abs(r.values[3][0] - a * math.sqrt(6) / 4) <= 1e-9


def _circumradius(V):
    V = np.asarray(V, np.float64)
    A = 2 * (V[1:] - V[0])
    b = (V[1:] ** 2).sum(1) - (V[0] ** 2).sum()
    if V.shape[0] == 3:
        n = np.cross(V[1] - V[0], V[2] - V[0])
        A = np.vstack([A, n])
        b = np.append(b, n @ V[0])
    c = np.linalg.solve(A, b)
    return c, np.linalg.norm(c - V[0])


@pytest.mark.parametrize("m", [5, 7, 11, 12])
def test_acute_simplex_approaches_circumradius_from_below(m):
    """R - (1/m) sqrt(sum |vi-vj|^2) <= f_P <= R for X = the vertices of an acute simplex."""
    V3 = np.array([[0, 0, 0], [1.0, 0.1, 0], [0.45, 0.9, 0.05]])
    V4 = np.array([[1.0, 0.9, 1.1], [1.0, -1.1, -0.9], [-1.0, 1.0, -1.05], [-0.95, -1.0, 1.0]])
    for V in (V3, V4):
        k = V.shape[0] - 1
        c, R = _circumradius(V)
        lam = np.linalg.lstsq(np.vstack([V.T, np.ones(k + 1)]), np.append(c, 1.0), rcond=None)[0]
        assert np.all(lam > 0)                                # circumcentre inside: acute
        S = _cx([list(range(k + 1))], k + 1)
        f = oracle.flood_values(V, V, S, m=m).values[k][0]
        bound = math.sqrt(sum(np.sum((V[i] - V[j]) ** 2) for i in range(k + 1) for j in range(i))) / m
        assert R - bound - 1e-12 <= f <= R + 1e-12


def test_triangle_value_bounded_by_minimal_enclosing_ball():
    """App. C: f(sigma) <= radius of the minimal enclosing ball of sigma when sigma ⊂ X."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        V = rng.standard_normal((3, 3))
        X = np.concatenate([V, rng.standard_normal((50, 3)) * 2])
        e = [np.linalg.norm(V[i] - V[j]) for i, j in ((0, 1), (1, 2), (0, 2))]
        a, b, c = sorted(e)
        obtuse = c * c >= a * a + b * b
        meb = c / 2 if obtuse else _circumradius(V)[1]
        f = oracle.flood_values(X, V, _cx([[0, 1, 2]], 3), m=9).values[2][0]
        assert f <= meb + 1e-12


def test_refinement_bound():
    """Theorem 3 with Lemma 1: m | m' => f_m <= f_m' <= f_m + (1/m) sqrt(sum |vi-vj|^2)."""
    X = data.torus_cloud(3000, seed=21)
    idx, _ = oracle.fps(X, 25)
    L = X[idx]
    cx = delaunay_complex(L)
    f4 = oracle.flood_values(X, L, cx.simplices, 4)
    f12 = oracle.flood_values(X, L, cx.simplices, 12)
    for k in range(1, 4):
        V = L[cx.simplices[k]].astype(np.float64)
        b = np.sqrt(sum(((V[:, i] - V[:, j]) ** 2).sum(1) for i in range(k + 1) for j in range(i))) / 4
        assert np.all(f4.values[k] <= f12.values[k] + 1e-12)
        assert np.all(f12.values[k] <= f4.values[k] + b + 1e-12)


def test_stability_in_X():
    """Theorem 1 (per simplex): moving every point of X by <= delta moves each f by <= delta."""
    X = data.sphere_cloud(2000, seed=8)
    idx, _ = oracle.fps(X, 30)
    L = X[idx]
    cx = delaunay_complex(L)
    rng = np.random.default_rng(9)
    delta = 0.01
    move = rng.standard_normal(X.shape)
    move *= delta * rng.uniform(0, 1, (X.shape[0], 1)) / np.linalg.norm(move, axis=1, keepdims=True)
    X2 = X.astype(np.float64) + move
    X2[idx] = X[idx]                       # keep L ⊂ X2
    a = oracle.flood_values(X, L, cx.simplices, 6)
    b = oracle.flood_values(X2, L, cx.simplices, 6)
    for k in range(1, 4):
        assert np.max(np.abs(a.values[k] - b.values[k])) <= delta + 1e-12


def test_masking_lemma_restricts_X_without_changing_values():
    """Lemma 2 (§4.2): X ∩ B_{sqrt2 r}(c) gives the same value as X (Ritter-style ball)."""
    X = data.torus_cloud(4000, seed=31)
    idx, _ = oracle.fps(X, 30)
    L = X[idx]
    cx = delaunay_complex(L)
    full = oracle.flood_values(X, L, cx.simplices, 6)
    X64 = X.astype(np.float64)
    rng = np.random.default_rng(2)
    for k in (1, 2, 3):
        for sid in rng.choice(cx.simplices[k].shape[0], 15, replace=False):
            c, r, rad = ritter_ball(L[cx.simplices[k][sid]])
            Xm = X64[np.linalg.norm(X64 - c, axis=1) <= rad]
            sub = [np.zeros((0, j + 1), np.int64) for j in range(k)] + [cx.simplices[k][[sid]]]
            v = oracle.flood_values(Xm, L, sub, 6).values[k][0]
            assert v == full.values[k][sid]


def test_face_values_never_exceed_coface_values():
    X = data.shape_mix_cloud(20000, seed=41)
    idx, _ = oracle.fps(X, 60)
    L = X[idx]
    cx = delaunay_complex(L)
    r = oracle.flood_values(X, L, cx.simplices, 6, method="kdtree")
    for k in range(1, 4):
        fac = r.values[k - 1][cx.facets[k]]
        assert np.all(fac.max(axis=1) <= r.values[k])


def test_full_grid_equals_interior_max_then_face_max():
    """App. A.1 identity: max over the full grid = max(interior samples, facet values)."""
    X = data.torus_cloud(5000, seed=51)
    idx, _ = oracle.fps(X, 40)
    L = X[idx].astype(np.float64)
    cx = delaunay_complex(L)
    m = 6
    full = oracle.flood_values(X, L, cx.simplices, m, method="kdtree")
    ind = KDIndex(X, "kdtree")
    for k in range(1, 4):
        comps = oracle.interior_compositions(m, k)
        V = L[cx.simplices[k]]
        P = np.einsum("fj,njd->nfd", comps / m, V)
        d, _ = ind.query(P.reshape(-1, 3))
        inner = d.reshape(V.shape[0], -1).max(axis=1)
        fac = full.values[k - 1][cx.facets[k]].max(axis=1)
        assert np.array_equal(np.maximum(inner, fac), full.values[k])


def test_kdtree_matches_brute_force():
    X = data.shape_mix_cloud(30000, seed=61)
    rng = np.random.default_rng(0)
    Q = rng.uniform(-5, 5, (3000, 3))
    d1, i1 = KDIndex(X, "brute").query(Q)
    d2, i2 = KDIndex(X, "kdtree").query(Q)
    assert np.allclose(d1, d2, rtol=0, atol=1e-12)
    assert np.mean(i1 == i2) > 0.999


@pytest.mark.parametrize("n_l", [8, 12])
def test_circle_edges_are_sagittas(n_l):
    """App. C.3: an edge along the circle floods at the sagitta 1 - cos(phi/2) of its arc."""
    n = 4096
    X = _circle(n)
    idx, _ = oracle.fps(X, n_l)
    order = np.argsort(idx)
    s = idx[order]
    edges = np.sort(np.stack([order, np.roll(order, -1)], axis=1), axis=1)
    arcs = np.diff(np.concatenate([s, [s[0] + n]])) * 2 * np.pi / n
    r = oracle.flood_values(X, X[idx], [np.zeros((0, 1), np.int64), edges], m=12, method="kdtree")
    assert np.allclose(r.values[1], 1 - np.cos(arcs / 2), rtol=0, atol=2e-7)


# ----------------------------------------------------------------------------- persistence

def _gf2_rank(M):
    M = M.copy() % 2
    r = 0
    rows, cols = M.shape
    for c in range(cols):
        piv = np.nonzero(M[r:, c])[0]
        if piv.size == 0:
            continue
        p = r + piv[0]
        M[[r, p]] = M[[p, r]]
        for q in np.nonzero(M[:, c])[0]:
            if q != r:
                M[q] ^= M[r]
        r += 1
        if r == rows:
            break
    return r


def test_diagrams_reproduce_betti_numbers():
    """beta_k(t) = #{(b,d) in dgm_k : b <= t < d}, with beta from GF(2) ranks of boundary maps."""
    X = data.sphere_cloud(600, seed=71)
    idx, _ = oracle.fps(X, 12)
    L = X[idx]
    cx = delaunay_complex(L)
    r = oracle.flood_values(X, L, cx.simplices, 4)
    vals = r.values
    dg = oracle.diagrams(cx.simplices, cx.facets, vals)
    for t in sorted(set(np.concatenate(vals).tolist())):
        alive = [np.nonzero(v <= t)[0] for v in vals]
        betti = []
        ranks = [0]
        for k in range(1, 4):
            rows = {int(a): i for i, a in enumerate(alive[k - 1])}
            B = np.zeros((len(alive[k - 1]), len(alive[k])), dtype=np.uint8)
            for j, s in enumerate(alive[k]):
                for f in cx.facets[k][s]:
                    B[rows[int(f)], j] = 1
            ranks.append(_gf2_rank(B) if B.size else 0)
        ranks.append(0)
        for k in range(3):
            betti.append(len(alive[k]) - ranks[k] - ranks[k + 1])
        for k in range(3):
            d = dg[k]
            count = int(np.sum((d[:, 0] <= t) & (t < d[:, 1])))
            assert count == betti[k], (t, k)


def test_circle_diagrams_closed_form():
    """App. C.3: dgm_0 = boundary sagittas (all but the one closing the cycle) + (0, inf);
    dgm_1 = {(largest boundary sagitta, ~1)}, death within Lemma 1's bound of 1."""
    n, n_l, m = 4096, 12, 12
    X = _circle(n)
    idx, _ = oracle.fps(X, n_l)
    order = np.argsort(idx)
    s = idx[order]
    arcs = np.diff(np.concatenate([s, [s[0] + n]])) * 2 * np.pi / n
    tris = [[order[0], order[i], order[i + 1]] for i in range(1, n_l - 1)]
    cx = complex_from_simplices([np.sort(np.array(tris), axis=1)], n_l)
    r = oracle.flood_values(X, X[idx], cx.simplices, m=m, method="kdtree")
    dg = oracle.diagrams(cx.simplices, cx.facets, r.values)
    sag = np.sort(1 - np.cos(arcs / 2))
    want0 = np.array([[0.0, v] for v in sag[:-1]] + [[0.0, np.inf]])
    assert oracle.bottleneck(dg[0], want0) <= 1e-6
    big = dg[1][(dg[1][:, 1] - dg[1][:, 0]) > 1e-4]
    assert big.shape[0] == 1
    assert abs(big[0, 0] - sag[-1]) <= 1e-6
    V = X[idx].astype(np.float64)
    bound = max(math.sqrt(sum(np.sum((V[t[i]] - V[t[j]]) ** 2) for i in range(3) for j in range(i))) / m
                for t in cx.simplices[2])
    assert 1 - bound <= big[0, 1] <= 1 + 1e-6


def test_bottleneck_known_cases():
    A = np.array([[0.0, 1.0]])
    assert oracle.bottleneck(A, np.array([[0.0, 1.2]])) == pytest.approx(0.2)
    assert oracle.bottleneck(A, np.zeros((0, 2))) == pytest.approx(0.5)
    assert oracle.bottleneck(np.array([[0.0, np.inf]]), np.array([[0.3, np.inf]])) == pytest.approx(0.3)
    assert oracle.bottleneck(np.array([[0.0, np.inf]]), np.zeros((0, 2))) == float("inf")
    rng = np.random.default_rng(3)
    D = [np.sort(rng.uniform(0, 1, (6, 2)), axis=1) for _ in range(3)]
    ab, bc, ac = oracle.bottleneck(D[0], D[1]), oracle.bottleneck(D[1], D[2]), oracle.bottleneck(D[0], D[2])
    assert ac <= ab + bc + 1e-12
    assert oracle.bottleneck(D[0], D[1]) == pytest.approx(oracle.bottleneck(D[1], D[0]))


def _bottleneck_brute(A, B):
    """Bottleneck distance by trying every bijection of A + diag(B) onto B + diag(A) (tiny diagrams)."""
    import itertools
    A = [tuple(p) for p in np.asarray(A, np.float64).reshape(-1, 2)]
    B = [tuple(p) for p in np.asarray(B, np.float64).reshape(-1, 2)]
    left = [("pt", p) for p in A] + [("diag", q) for q in B]
    right = [("pt", q) for q in B] + [("diag", p) for p in A]

    def cost(a, b):
        if a[0] == "pt" and b[0] == "pt":
            p, q = a[1], b[1]
            if np.isinf(p[1]) != np.isinf(q[1]):
                return np.inf
            return max(abs(p[0] - q[0]), 0.0 if np.isinf(p[1]) else abs(p[1] - q[1]))
        if a[0] == "pt":                       # a point to the diagonal
            return np.inf if np.isinf(a[1][1]) else (a[1][1] - a[1][0]) / 2
        if b[0] == "pt":
            return np.inf if np.isinf(b[1][1]) else (b[1][1] - b[1][0]) / 2
        return 0.0
    return min(max([cost(a, b) for a, b in zip(left, perm)], default=0.0)
               for perm in itertools.permutations(right))


def test_bottleneck_and_its_threshold_test_match_brute_force():
    """bottleneck = the min over bijections of the largest L-inf move (§2), diagonal allowed;
    bottleneck_within(eps) is true exactly from that value on."""
    rng = np.random.default_rng(11)
    for trial in range(40):
        na, nb = rng.integers(0, 4), rng.integers(0, 4)
        A = np.sort(rng.uniform(0, 1, (na, 2)), axis=1)
        B = np.sort(rng.uniform(0, 1, (nb, 2)), axis=1)
        if trial % 3 == 0:                              # one essential class on each side
            A = np.vstack([A, [[rng.uniform(0, 1), np.inf]]])
            B = np.vstack([B, [[rng.uniform(0, 1), np.inf]]])
        want = _bottleneck_brute(A, B)
        got = oracle.bottleneck(A, B)
        assert got == pytest.approx(want, abs=1e-12), (trial, got, want)
        assert oracle.bottleneck_within(A, B, want + 1e-12)
        if want > 1e-9:
            assert not oracle.bottleneck_within(A, B, want - 1e-9)


def test_persistence_pairs_partition_the_simplices():
    """Every simplex is created-and-killed in exactly one pair or is essential; a pair joins a
    k-simplex to a (k+1)-simplex later in the filtration order; the essential classes of a
    triangulated 3-ball are one component (beta = 1, 0, 0, 0)."""
    X = data.sphere_cloud(800, seed=72)
    idx, _ = oracle.fps(X, 40)
    L = X[idx]
    cx = delaunay_complex(L)
    vals = oracle.flood_values(X, L, cx.simplices, 4).values
    pairs, essential = oracle.persistence_pairs(cx.simplices, cx.facets, vals)
    order, _ = oracle.persistence.filtration_order(cx.simplices, vals)
    pos = {kr: i for i, kr in enumerate(order)}
    seen = [b for b, _ in pairs] + [d for _, d in pairs] + list(essential)
    assert len(seen) == len(set(seen)) == sum(cx.counts)
    for b, d in pairs:
        assert d[0] == b[0] + 1 and pos[b] < pos[d]
    assert [sum(1 for e in essential if e[0] == k) for k in range(4)] == [1, 0, 0, 0]


# ----------------------------------------------------------------------------- gradient

def test_analytic_gradient_matches_central_differences():
    X = data.jitter(data.torus_cloud(600, seed=81), amp=1e-6, seed=82)
    idx, _ = oracle.fps(X, 16)
    L = X[idx].copy()
    cx = delaunay_complex(L)
    gamma = data.upstream_gradients(cx.counts, seed=83)
    m = 5
    res = oracle.flood_values(X, L, cx.simplices, m, method="brute")
    dX, dL = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=res)
    rng = np.random.default_rng(4)
    nzX = np.argwhere(np.abs(dX) > 0)
    probes = [("X", int(a), int(b)) for a, b in nzX[rng.choice(len(nzX), 40, replace=False)]]
    probes += [("L", int(a), int(b)) for a in rng.choice(L.shape[0], 10) for b in [int(rng.integers(3))]]
    probes += [("X", int(a), 1) for a in rng.choice(X.shape[0], 10)]
    fd, kink, _ = oracle.finite_difference(X, L, cx.simplices, m, gamma, probes, h=1e-6, method="brute")
    an = np.array([dX[r, c] if w == "X" else dL[r, c] for (w, r, c) in probes])
    ok = ~kink
    assert ok.sum() >= 40
    assert np.allclose(fd[ok], an[ok], rtol=1e-3, atol=1e-5)


# ----------------------------------------------------------------------------- faces

def test_faces_of_one_and_two_tetrahedra():
    tri, edg = oracle.faces_by_definition([[0, 1, 2, 3]])
    assert tri.shape == (4, 3) and edg.shape == (6, 2)
    tri, edg = oracle.faces_by_definition([[0, 1, 2, 3], [1, 2, 3, 4]])   # sharing triangle 123
    assert tri.shape == (7, 3) and edg.shape == (9, 2)
    f = oracle.facet_rows(np.array([[0, 1, 2, 3]]), tri)
    assert [tuple(tri[r]) for r in f[0]] == [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]


def test_faces_of_a_delaunay_ball():
    """Del of generic points is a triangulated 3-ball: Euler characteristic 1, and the
    triangles used by one tetrahedron are exactly Qhull's convex hull facets."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(7)
    P = rng.standard_normal((300, 3))
    d = Delaunay(P)
    tets = np.sort(d.simplices, axis=1)
    tri, edg = oracle.faces_by_definition(tets)
    assert P.shape[0] - edg.shape[0] + tri.shape[0] - tets.shape[0] == 1
    use = np.bincount(oracle.facet_rows(tets, tri).ravel(), minlength=tri.shape[0])
    assert set(np.unique(use)) <= {1, 2}
    hull = {tuple(sorted(r)) for r in d.convex_hull.tolist()}
    assert {tuple(r) for r in tri[use == 1].tolist()} == hull
    assert 4 * tets.shape[0] == 2 * np.count_nonzero(use == 2) + len(hull)


# ----------------------------------------------------------------------------- landmarks off X (§3: L need not be in X)

def test_vertex_off_X_is_its_distance():
    X = np.array([[0.0, 0.0, 0.0], [10.0, 0.0, 0.0]])
    L = np.array([[3.0, 4.0, 0.0]])
    r = oracle.flood_values(X, L, [np.zeros((1, 1), np.int64)], m=4)
    assert abs(r.values[0][0] - 5.0) <= 1e-12


@pytest.mark.parametrize("m", [2, 4, 7])
def test_edge_off_X_attained_at_a_vertex(m):
    """X = {origin}, edge from (-1,1,0) to (1,1,0): d(p, X) = sqrt(x^2 + 1) peaks at the ends."""
    X = np.zeros((1, 3))
    L = np.array([[-1.0, 1.0, 0.0], [1.0, 1.0, 0.0]])
    r = oracle.flood_values(X, L, [np.arange(2)[:, None], np.array([[0, 1]])], m=m)
    assert abs(r.values[1][0] - math.sqrt(2.0)) <= 1e-12
    assert np.allclose(r.values[0], math.sqrt(2.0), rtol=0, atol=1e-12)


def test_values_are_1_lipschitz_in_the_landmarks():
    """Every sample p = sum lambda_j v_j moves by at most max_j |dv_j|, so f moves by at most that."""
    X = data.torus_cloud(4000, seed=141)
    idx, _ = oracle.fps(X, 30)
    rng = np.random.default_rng(142)
    L = X[idx].astype(np.float64) + rng.uniform(-0.02, 0.02, (30, 3))
    cx = delaunay_complex(L)
    delta = 0.01
    step = rng.standard_normal(L.shape)
    step *= delta / np.linalg.norm(step, axis=1, keepdims=True)
    a = oracle.flood_values(X, L, cx.simplices, 5, method="kdtree")
    b = oracle.flood_values(X, L + step, cx.simplices, 5, method="kdtree")
    for k in range(4):
        assert np.max(np.abs(a.values[k] - b.values[k])) <= delta + 1e-12
    assert np.all(a.values[0] > 0)


def test_analytic_gradient_with_landmarks_off_X():
    X = data.jitter(data.torus_cloud(600, seed=151), amp=1e-6, seed=152).astype(np.float64)
    idx, _ = oracle.fps(X, 14)
    rng = np.random.default_rng(153)
    L = X[idx] + rng.uniform(-0.05, 0.05, (14, 3))
    cx = delaunay_complex(L)
    gamma = data.upstream_gradients(cx.counts, seed=154)
    m = 4
    res = oracle.flood_values(X, L, cx.simplices, m, method="brute")
    assert any(np.any(res.argmax_sample[k] >= 0) for k in range(4))
    dX, dL = oracle.analytic_gradient(X, L, cx.simplices, m, gamma, result=res)
    nzX = np.argwhere(np.abs(dX) > 0)
    probes = [("X", int(a), int(b)) for a, b in nzX[rng.choice(len(nzX), 30, replace=False)]]
    probes += [("L", int(a), int(rng.integers(3))) for a in range(14)]
    fd, kink, _ = oracle.finite_difference(X, L, cx.simplices, m, gamma, probes, h=1e-6, method="brute")
    an = np.array([dX[r, c] if w == "X" else dL[r, c] for (w, r, c) in probes])
    ok = ~kink
    assert ok.sum() >= 30
    assert np.allclose(fd[ok], an[ok], rtol=1e-3, atol=1e-5)


def _golden_counts():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "grid_counts_sec5_3.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return [tuple(int(v) for v in r) for r in rows]


def test_grid_counts_printed_in_the_paper():
    """§5.3: 20 points per edge -> 210 per triangle, 1540 per tetrahedron (golden fixture)."""
    for per_edge, per_tri, per_tet in _golden_counts():
        m = per_edge - 1
        assert oracle.compositions(m, 1).shape[0] == per_edge
        assert oracle.compositions(m, 2).shape[0] == per_tri
        assert oracle.compositions(m, 3).shape[0] == per_tet
        # the full grid is the interior grids of all faces: vertices, edges, triangles, itself
        assert 4 + 6 * oracle.interior_count(m, 1) + 4 * oracle.interior_count(m, 2) + \
            oracle.interior_count(m, 3) == per_tet
