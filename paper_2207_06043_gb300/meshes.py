"""Seeded capsule meshes and placements: the input side of ``ibl_add_capsule``.

Icospheres (12, 42, 162, 642, 2562, ... vertices) with outward
counter-clockwise triangles, analytic ellipsoids built from them, a seeded
rotation, and rejection sampling of non-overlapping capsule centres.  No
membrane or immersed-boundary arithmetic lives here.
"""
from __future__ import annotations

import math

import numpy as np


def _splitmix64(state):
    """SplitMix64 step on a Python int; returns (new_state, value)."""
    state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return state, z ^ (z >> 31)


class SplitMix64:
    """Counter-based generator used for every seeded draw of the workloads."""

    def __init__(self, seed: int):
        self.state = int(seed) & 0xFFFFFFFFFFFFFFFF

    def next_u64(self) -> int:
        self.state, v = _splitmix64(self.state)
        return v

    def uniform(self, lo=0.0, hi=1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))

    def unit_vector(self) -> np.ndarray:
        z = self.uniform(-1.0, 1.0)
        a = self.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        return np.array([s * math.cos(a), s * math.sin(a), z])


def icosphere(subdivisions: int):
    """Unit icosphere: (vertices (V,3) float64, triangles (T,3) int32), outward CCW."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdivisions):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts)
    T = np.array(faces, dtype=np.int32)
    # orient outward
    cen = V[T].mean(axis=1)
    nrm = np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]])
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return V, T


def subdivisions_for(n_vertices: int) -> int:
    for s in range(8):
        if 10 * 4 ** s + 2 == n_vertices:
            return s
    raise ValueError(f"no icosphere has {n_vertices} vertices")


def random_rotation(rng: SplitMix64) -> np.ndarray:
    """Uniform random rotation matrix (from a random unit quaternion)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    q = np.array([math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
                  math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
                  math.sqrt(u1) * math.sin(2 * math.pi * u3),
                  math.sqrt(u1) * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def sphere_mesh(n_vertices: int, diameter: float, centre, rng: SplitMix64 | None = None):
    V, T = icosphere(subdivisions_for(n_vertices))
    if rng is not None:
        V = V @ random_rotation(rng).T
    return V * (diameter / 2.0) + np.asarray(centre, dtype=np.float64), T


def ellipsoid_mesh(n_vertices: int, semi_axes, centre):
    V, T = icosphere(subdivisions_for(n_vertices))
    return V * np.asarray(semi_axes, dtype=np.float64) + np.asarray(centre, dtype=np.float64), T


def place_capsules(rng: SplitMix64, n: int, diameter: float, x_range, yc, zc, duct_half,
                   margin=2.0, min_gap=2.0, max_tries=200000):
    """Rejection-sample n centres in x_range inside a square duct centred at
    (yc, zc) with half side duct_half, each at least diameter/2 + margin from
    the duct walls and diameter + min_gap from every other centre."""
    r = diameter / 2.0
    lim = duct_half - r - margin
    if lim < 0:
        raise ValueError("capsule does not fit in the duct")
    lo = x_range[0] + r + margin
    hi = x_range[1] - r - margin
    centres = []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place capsules without overlap")
        c = np.array([rng.uniform(lo, hi), yc + rng.uniform(-lim, lim), zc + rng.uniform(-lim, lim)])
        if all(np.linalg.norm(c - o) >= diameter + min_gap for o in centres):
            centres.append(c)
    return np.array(centres)


def fibonacci_sphere(n_vertices: int):
    """Unit sphere through n_vertices points on the Fibonacci spiral, triangulated
    as their convex hull (every point is a hull vertex), outward CCW: a closed
    mesh with any vertex count (2 n - 4 triangles)."""
    from scipy.spatial import ConvexHull
    n = int(n_vertices)
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / n
    phi = math.pi * (3.0 - math.sqrt(5.0)) * i
    s = np.sqrt(1.0 - z * z)
    P = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    T = ConvexHull(P).simplices.astype(np.int32)
    # orient outward: the triangle normal points away from the origin
    a, b, c = P[T[:, 0]], P[T[:, 1]], P[T[:, 2]]
    flip = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    return P, T


def sphere_mesh_n(n_vertices: int, diameter: float, centre, rng: SplitMix64):
    """Fibonacci sphere of n_vertices vertices, scaled to `diameter`, randomly
    rotated and placed at `centre`."""
    V, T = fibonacci_sphere(n_vertices)
    R = random_rotation(rng)
    return (V @ R.T) * (0.5 * diameter) + np.asarray(centre, dtype=np.float64)[None, :], T


def tube_mesh(x0: float, x1: float, radius: float, yc: float, zc: float, h: float, periodic_x: bool = False):
    """Open circular tube of the given radius around the line (y, z) = (yc, zc),
    from x0 to x1, triangulated with edges of about h: rings of
    ceil(2 pi radius / h) vertices about h sqrt(3)/2 apart, every other ring
    turned by half a step.  periodic_x: an even number of ring spacings, so
    that the ring at x1 repeats the one at x0 shifted by x1 - x0 (a tube that
    continues across a periodic x axis of that length).  A fixed-wall surface:
    its triangle centroids are the wall markers."""
    n_t = max(8, int(math.ceil(2.0 * math.pi * radius / h)))
    length = float(x1 - x0)
    n_b = max(2, int(math.ceil(length / (h * math.sqrt(3.0) / 2.0))))
    if periodic_x and n_b % 2:
        n_b += 1
    dxr = length / n_b
    k = np.arange(n_b + 1)[:, None]
    j = np.arange(n_t)[None, :]
    th = 2.0 * math.pi * (j + 0.5 * (k % 2)) / n_t
    X = np.broadcast_to(x0 + dxr * k, th.shape)
    V = np.stack([X, yc + radius * np.cos(th), zc + radius * np.sin(th)], axis=-1).reshape(-1, 3)
    tris = []
    for r in range(n_b):
        for t in range(n_t):
            t2 = (t + 1) % n_t
            a, b = r * n_t + t, r * n_t + t2
            c, d = (r + 1) * n_t + t, (r + 1) * n_t + t2
            if r % 2 == 0:
                tris += [(a, b, c), (b, d, c)]
            else:
                tris += [(a, b, d), (a, d, c)]
    return V.astype(np.float64), np.array(tris, dtype=np.int32)
