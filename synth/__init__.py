"""Seeded synthetic inputs: meshes, noise and probe vectors.

This module is shared by the FP64 oracle tests, the GPU parity tests and the
benchmark. It holds no arithmetic of the tangent-point method itself (no
kernel, energy, operator or solver): only mesh generators, seeded
perturbations and seeded random vectors.

Workloads (sizes follow the benchmark configurations of the method's
hot path):

* ``icosphere_l3``   -- icosphere level 3 (642 vertices, 1280 triangles,
  radius 1), every vertex displaced by i.i.d. N(0, 0.01^2) per coordinate.
* ``torus_20k``      -- torus R=1, r=0.3 on a 200 x 50 vertex grid
  (10,000 vertices, 20,000 triangles), N(0, 0.005^2) noise.
* ``linked_tori_50k`` -- two tori R=1, r=0.25, each a 250 x 50 grid
  (25,000 triangles each); the second is rotated 90 degrees about x and
  translated by (1, 0, 0), so the two centre lines form a Hopf link.
* ``icosphere_l8``   -- icosphere level 8 (655,362 vertices, 1,310,720
  triangles) with a radial bump 0.05 g / max|g|, g a random combination of
  real spherical harmonics of degree 1..8.

Static-obstacle scene:

* ``ball_in_torus_hole`` -- a sphere of radius 0.5 (icosphere level 5,
  10,242 vertices, 20,480 triangles, no noise) centred at the origin, i.e.
  in the hole of ``torus_20k`` (hole radius 0.7): the obstacle mesh of the
  obstacle benchmark, with ``torus_20k`` as the moving surface.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "icosphere", "torus", "linked_tori", "gaussian_noise", "sh_bumps",
    "vertex_vectors", "workload", "WORKLOADS", "small_mesh", "obstacle", "OBSTACLES",
]


# ---------------------------------------------------------------------------
# mesh generators
# ---------------------------------------------------------------------------

def _orient_outward(V, F):
    """Flip faces whose normal points towards the centroid of the mesh
    (valid for star-shaped closed meshes such as the icosahedron)."""
    c = V.mean(axis=0)
    a, b, d = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    n = np.cross(b - a, d - a)
    s = np.einsum("ij,ij->i", n, (a + b + d) / 3.0 - c)
    F = F.copy()
    flip = s < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return F


def icosphere(level: int, radius: float = 1.0):
    """Midpoint-subdivided regular icosahedron, projected to a sphere.

    Returns (V float64 [nv,3], F int32 [nf,3]); faces are counter-clockwise
    seen from outside. nv = 10*4^level + 2, nf = 20*4^level.
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    V = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    F = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    F = _orient_outward(V, F)
    for _ in range(level):
        nv = V.shape[0]
        e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], axis=0)
        key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
        uniq, inv = np.unique(key, return_inverse=True)
        i0, i1 = uniq // nv, uniq % nv
        mid = 0.5 * (V[i0] + V[i1])
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = F.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        a, b, c = F[:, 0], F[:, 1], F[:, 2]
        F = np.concatenate([
            np.stack([a, m01, m20], 1), np.stack([b, m12, m01], 1),
            np.stack([c, m20, m12], 1), np.stack([m01, m12, m20], 1)], axis=0)
        V = np.concatenate([V, mid], axis=0)
    return V * radius, F.astype(np.int32)


def torus(n_major: int, n_minor: int, R: float, r: float):
    """Torus on an n_major x n_minor vertex grid, each quad split on the
    same diagonal; outward-oriented counter-clockwise faces.
    nv = n_major*n_minor, nf = 2*nv."""
    i = np.arange(n_major)
    j = np.arange(n_minor)
    u = 2.0 * np.pi * i / n_major
    v = 2.0 * np.pi * j / n_minor
    U, W = np.meshgrid(u, v, indexing="ij")
    V = np.stack([(R + r * np.cos(W)) * np.cos(U),
                  (R + r * np.cos(W)) * np.sin(U),
                  r * np.sin(W)], axis=-1).reshape(-1, 3)
    I, J = np.meshgrid(i, j, indexing="ij")
    a = I * n_minor + J
    b = ((I + 1) % n_major) * n_minor + J
    c = ((I + 1) % n_major) * n_minor + (J + 1) % n_minor
    d = I * n_minor + (J + 1) % n_minor
    F = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3),
                        np.stack([a, c, d], -1).reshape(-1, 3)], axis=0)
    # orientation: the normal must point away from the tube's centre line
    X = V[F].mean(axis=1)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    ang = np.arctan2(X[:, 1], X[:, 0])
    centre = np.stack([R * np.cos(ang), R * np.sin(ang), np.zeros_like(ang)], -1)
    flip = np.einsum("ij,ij->i", n, X - centre) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F.astype(np.int32)


def linked_tori(n_major: int = 250, n_minor: int = 50, R: float = 1.0,
                r: float = 0.25, offset: float = 1.0):
    """Two interlinked tori: the second is the first rotated 90 degrees about
    the x axis and translated by (offset, 0, 0)."""
    V1, F1 = torus(n_major, n_minor, R, r)
    rot = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])
    V2 = V1 @ rot.T + np.array([offset, 0.0, 0.0])
    V = np.concatenate([V1, V2], axis=0)
    F = np.concatenate([F1, F1 + V1.shape[0]], axis=0)
    return V, F.astype(np.int32)


# ---------------------------------------------------------------------------
# seeded perturbations and vectors
# ---------------------------------------------------------------------------

def gaussian_noise(V, sigma: float, seed: int):
    """i.i.d. N(0, sigma^2) displacement of every coordinate."""
    rng = np.random.default_rng(seed)
    return V + sigma * rng.standard_normal(V.shape)


def _real_sph_harm(lmax: int, theta, phi):
    """Orthonormal real spherical harmonics Y_lm for 1 <= l <= lmax, as a list
    of arrays, using the standard three-term recurrence of the normalised
    associated Legendre functions (theta = polar angle)."""
    x = np.cos(theta)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    # Pbar[l][m]: fully normalised associated Legendre functions
    P = {}
    P[(0, 0)] = np.full_like(x, 1.0 / np.sqrt(4.0 * np.pi))
    for m in range(1, lmax + 1):
        P[(m, m)] = -np.sqrt((2.0 * m + 1.0) / (2.0 * m)) * sx * P[(m - 1, m - 1)]
    for m in range(0, lmax):
        P[(m + 1, m)] = np.sqrt(2.0 * m + 3.0) * x * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            a = np.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = np.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            P[(l, m)] = a * (x * P[(l - 1, m)] - b * P[(l - 2, m)])
    out = []
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            if m == 0:
                out.append(P[(l, 0)])
            elif m > 0:
                out.append(np.sqrt(2.0) * P[(l, m)] * np.cos(m * phi))
            else:
                out.append(np.sqrt(2.0) * P[(l, -m)] * np.sin(-m * phi))
    return out


def sh_bumps(V, lmax: int, amplitude: float, seed: int):
    """Radial bump f -> f * (1 + amplitude * g / max|g|) with
    g = sum_{l=1..lmax} sum_m c_lm Y_lm, c_lm ~ N(0,1) seeded."""
    rng = np.random.default_rng(seed)
    rad = np.linalg.norm(V, axis=1)
    theta = np.arccos(np.clip(V[:, 2] / rad, -1.0, 1.0))
    phi = np.arctan2(V[:, 1], V[:, 0])
    Y = _real_sph_harm(lmax, theta, phi)
    c = rng.standard_normal(len(Y))
    g = np.zeros_like(rad)
    for ci, yi in zip(c, Y):
        g += ci * yi
    g /= np.abs(g).max()
    return V * (1.0 + amplitude * g)[:, None]


def vertex_vectors(nv: int, k: int, seed: int):
    """Seeded N(0,1) per-vertex vectors, shape [nv, k], float64."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nv, k))


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def _icosphere_l3():
    V, F = icosphere(3)
    return gaussian_noise(V, 0.01, 1), F


def _torus_20k():
    V, F = torus(200, 50, 1.0, 0.3)
    return gaussian_noise(V, 0.005, 2), F


def _linked_tori_50k():
    return linked_tori(250, 50, 1.0, 0.25, 1.0)


def _icosphere_l8():
    V, F = icosphere(8)
    return sh_bumps(V, 8, 0.05, 505), F


WORKLOADS = {
    "icosphere_l3": _icosphere_l3,
    "torus_20k": _torus_20k,
    "linked_tori_50k": _linked_tori_50k,
    "icosphere_l8": _icosphere_l8,
}


def workload(name: str):
    """(V float64 [nv,3], F int32 [nf,3]) of a named workload."""
    return WORKLOADS[name]()


def _ball_in_torus_hole():
    return icosphere(5, 0.5)


OBSTACLES = {
    "ball_in_torus_hole": _ball_in_torus_hole,
}


def obstacle(name: str):
    """(V float64 [nv,3], F int32 [nf,3]) of a named static obstacle mesh."""
    return OBSTACLES[name]()


def small_mesh(kind: str, seed: int = 7):
    """Small meshes for the CPU pins and the ragged-size parity cases."""
    if kind == "tetra":
        V = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
        F = _orient_outward(V, np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]]))
        return V, F.astype(np.int32)
    if kind == "octa":
        V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
                     dtype=np.float64)
        F = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
                      [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]])
        return V, _orient_outward(V, F).astype(np.int32)
    if kind.startswith("ico"):
        lvl = int(kind[3:])
        V, F = icosphere(lvl)
        return gaussian_noise(V, 0.01, seed), F
    if kind.startswith("torus"):
        a, b = (int(x) for x in kind[5:].split("x"))
        V, F = torus(a, b, 1.0, 0.3)
        return gaussian_noise(V, 0.005, seed), F
    raise KeyError(kind)
