"""Seeded synthetic point clouds shaped like the 3D workloads of the Flood complex paper.

This module is the ONLY code shared by the CUDA path and the oracle: it draws
coordinates and nothing else. It holds none of the method's arithmetic (no
distances, no samples, no flood values), only numpy's PCG64 generator in FP64
followed by one cast to float32.

The paper's own datasets (corals, virus, rocks, swisscheese files; App. A.4)
are not available, so these generators stand in for them at the sizes of the
workloads described in the paper's experiments (§5, App. A.4, App. B).

Workloads:
  sphere_cloud      unit sphere + isotropic Gaussian noise (10,000 points)
  torus_cloud       torus R=1, r=0.3, uniform in angles, + Gaussian noise (1M)
  shape_mix_cloud   union of 8 random surfaces in [-4,4]^3 (5M)
  swisscheese_cloud uniform in [0,5]^3 minus disjoint balls (§5.3 synthetic data)
  serving_sizes     log-uniform cloud sizes for the batched serving workload
  random_barycentric  uniform random barycentric coordinates (random P_sigma)
  annulus_cloud     planar annulus (ambient dimension 2), embedded at z = 0
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "sphere_cloud",
    "torus_cloud",
    "shape_mix_cloud",
    "swisscheese_cloud",
    "serving_sizes",
    "poisson_arrivals",
    "jitter",
    "upstream_gradients",
    "random_barycentric",
    "annulus_cloud",
    "embed_planar",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def sphere_cloud(n: int = 10_000, noise: float = 0.01, seed: int = 1) -> np.ndarray:
    """x = g/|g| + noise * n with g, n ~ N(0, I3)."""
    rng = _rng(seed)
    g = rng.standard_normal((n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return _f32(g + noise * rng.standard_normal((n, 3)))


def torus_cloud(n: int = 1_000_000, R: float = 1.0, r: float = 0.3,
                noise: float = 0.005, seed: int = 2) -> np.ndarray:
    """Torus surface, angles u, v ~ U[0, 2pi) (uniform in angles), + N(0, noise^2)."""
    rng = _rng(seed)
    u = rng.uniform(0.0, 2 * np.pi, n)
    v = rng.uniform(0.0, 2 * np.pi, n)
    x = np.stack([(R + r * np.cos(v)) * np.cos(u),
                  (R + r * np.cos(v)) * np.sin(u),
                  r * np.sin(v)], axis=1)
    return _f32(x + noise * rng.standard_normal((n, 3)))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _sphere_surface(rng, n, s):
    g = rng.standard_normal((n, 3))
    return s * g / np.linalg.norm(g, axis=1, keepdims=True)


def _torus_surface(rng, n, s):
    R, r = s, 0.3 * s
    out = np.empty((0, 3))
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        u = rng.uniform(0, 2 * np.pi, m)
        v = rng.uniform(0, 2 * np.pi, m)
        keep = rng.uniform(0, 1, m) < (R + r * np.cos(v)) / (R + r)
        u, v = u[keep], v[keep]
        p = np.stack([(R + r * np.cos(v)) * np.cos(u),
                      (R + r * np.cos(v)) * np.sin(u),
                      r * np.sin(v)], axis=1)
        out = np.concatenate([out, p])
    return out[:n]


def _ellipsoid_surface(rng, n, axes):
    # Area-uniform by rejection: sample the unit sphere, map by diag(axes), and
    # accept with probability proportional to the local area stretch.
    a = np.asarray(axes)
    out = np.empty((0, 3))
    amax = np.prod(a) / a.min()
    while out.shape[0] < n:
        m = 2 * (n - out.shape[0]) + 16
        g = rng.standard_normal((m, 3))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        stretch = np.prod(a) * np.sqrt(((g / a) ** 2).sum(axis=1))
        keep = rng.uniform(0, 1, m) < stretch / amax
        out = np.concatenate([out, g[keep] * a])
    return out[:n]


def _patch_surface(rng, n, s):
    uv = rng.uniform(-s, s, (n, 2))
    return np.concatenate([uv, np.zeros((n, 1))], axis=1)


def _shape_area(kind, s, axes):
    if kind == "sphere":
        return 4 * np.pi * s * s
    if kind == "torus":
        return 4 * np.pi ** 2 * s * (0.3 * s)
    if kind == "ellipsoid":
        a, b, c = axes
        p = 1.6075  # Knud Thomsen's approximation; only used to apportion points
        return 4 * np.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3) ** (1 / p)
    return (2 * s) ** 2


def shape_mix_cloud(n: int = 5_000_000, n_shapes: int = 8, noise: float = 0.01,
                    seed: int = 3) -> np.ndarray:
    """Union of random surfaces (sphere / torus / ellipsoid shell / planar patch).

    Centres ~ U[-4,4]^3, scales ~ U[0.5,2], uniform random rotations, points
    apportioned to shapes by surface area, then N(0, noise^2) per coordinate.
    """
    rng = _rng(seed)
    kinds = ["sphere", "torus", "ellipsoid", "patch"]
    shapes = []
    for _ in range(n_shapes):
        kind = kinds[rng.integers(0, 4)]
        c = rng.uniform(-4, 4, 3)
        s = rng.uniform(0.5, 2.0)
        axes = (s, s * rng.uniform(0.5, 1.0), s * rng.uniform(0.5, 1.0))
        Rm = _random_rotation(rng)
        shapes.append((kind, c, s, axes, Rm))
    areas = np.array([_shape_area(k, s, ax) for k, _, s, ax, _ in shapes])
    counts = np.floor(n * areas / areas.sum()).astype(np.int64)
    counts[: n - counts.sum()] += 1
    parts = []
    for (kind, c, s, axes, Rm), cnt in zip(shapes, counts):
        if kind == "sphere":
            p = _sphere_surface(rng, cnt, s)
        elif kind == "torus":
            p = _torus_surface(rng, cnt, s)
        elif kind == "ellipsoid":
            p = _ellipsoid_surface(rng, cnt, axes)
        else:
            p = _patch_surface(rng, cnt, s)
        parts.append(p @ Rm.T + c)
    x = np.concatenate(parts)
    x = x[rng.permutation(n)]
    return _f32(x + noise * rng.standard_normal((n, 3)))


def swisscheese_cloud(n: int = 1_000_000, n_holes: int = 10, seed: int = 6, dim: int = 3) -> np.ndarray:
    """Uniform points in [0,5]^dim minus n_holes disjoint balls, radii ~ U[0.1,0.5] (§5.3).

    dim = 3 is the swisscheese data set; dim in {2, 4, 5} gives the
    swisscheese-like clouds of the scaling study in the ambient dimension
    (§5.3, Fig. 4c: |X| = 1M, |L| = 1k).
    """
    rng = _rng(seed)
    centres, radii = [], []
    while len(centres) < n_holes:
        r = rng.uniform(0.1, 0.5)
        c = rng.uniform(r, 5 - r, dim)
        if all(np.linalg.norm(c - c2) > r + r2 for c2, r2 in zip(centres, radii)):
            centres.append(c)
            radii.append(r)
    out = np.empty((0, dim))
    C, Rr = np.array(centres), np.array(radii)
    while out.shape[0] < n:
        m = int(1.2 * (n - out.shape[0])) + 16
        p = rng.uniform(0, 5, (m, dim))
        inside = (np.linalg.norm(p[:, None, :] - C[None], axis=2) < Rr).any(axis=1)
        out = np.concatenate([out, p[~inside]])
    return _f32(out[:n])


def serving_sizes(n_clouds: int = 512, lo: int = 2_000, hi: int = 200_000, seed: int = 4) -> np.ndarray:
    """Cloud sizes log-uniform in [lo, hi] for the batched serving workload."""
    rng = _rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n_clouds)).astype(np.int64)


def poisson_arrivals(n: int, rate: float, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream with the given rate."""
    rng = _rng(seed + 1_000_003)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def jitter(x: np.ndarray, amp: float = 1e-6, seed: int = 5) -> np.ndarray:
    """x + U[-amp, amp] per coordinate (breaks exact ties)."""
    rng = _rng(seed)
    return _f32(x.astype(np.float64) + rng.uniform(-amp, amp, x.shape))


def upstream_gradients(sizes, seed: int = 5) -> list:
    """gamma ~ N(0,1) float32 per simplex, one array per dimension."""
    rng = _rng(seed + 17)
    return [_f32(rng.standard_normal(int(s))) for s in sizes]


def random_barycentric(n_simplices: int, n_samples: int, k: int, seed: int = 7) -> np.ndarray:
    """(n_simplices, n_samples, k+1) float32 barycentric coordinates, uniform on
    the k-simplex and independent per simplex (the random P_sigma of §4.1 and
    Lemma 4): normalised unit exponentials, i.e. a flat Dirichlet draw."""
    rng = _rng(seed + 1009 * (k + 1))
    e = rng.exponential(1.0, (int(n_simplices), int(n_samples), k + 1))
    return _f32(e / e.sum(axis=2, keepdims=True))


def embed_planar(xy: np.ndarray) -> np.ndarray:
    """(n, 2) planar points as (n, 3) float32 with z = 0 (ambient dimension 2)."""
    xy = np.asarray(xy, dtype=np.float64)
    return _f32(np.concatenate([xy, np.zeros((xy.shape[0], 1))], axis=1))


def annulus_cloud(n: int = 20_000, r_in: float = 0.6, r_out: float = 1.0, seed: int = 8) -> np.ndarray:
    """Points uniform (by area) in a planar annulus, embedded at z = 0, float32 (n, 3)."""
    rng = _rng(seed)
    r = np.sqrt(rng.uniform(r_in * r_in, r_out * r_out, n))
    t = rng.uniform(0.0, 2.0 * np.pi, n)
    return embed_planar(np.stack([r * np.cos(t), r * np.sin(t)], axis=1))
