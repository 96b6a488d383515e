"""Pins of the oracle's marker-based wall tagging (Section "Boundary conditions
on fixed bodies", Eq. qbouzidi; oracle/walls.py): a single marker worked by
hand, a brute-force restatement on tiny random inputs (periodic axes and
pre-tagged solid nodes included), and the steady flow through a tube whose
wall is given only by its triangulation."""
import math

import numpy as np

from oracle import lattice as L
from oracle import walls as Wl
from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms

SQ2 = math.sqrt(2.0)


def test_single_marker_by_hand():
    """One triangle with centroid L = (2.2, 3.1, 1.9) in a 6x6x5 box: its cell
    is node s = (2, 3, 2) (2.7, 3.6, 2.4 rounded down), the only solid node;
    the 18 nodes s - e_i are the boundary nodes, each with one link (toward
    s), q = |s - e_i - L| / |e_i| clipped to 1."""
    V = np.array([[2.2, 3.1, 1.9], [2.5, 3.1, 1.9], [1.9, 3.1, 1.9]])
    tag, node, dirs, q = Wl.voxelise_markers(V, [[0, 1, 2]], (6, 6, 5))
    s = 2 + 6 * (3 + 6 * 2)
    assert tag.sum() == 1 and tag[s] == 1
    assert len(node) == 18
    got = {int(d): float(qq) for d, qq in zip(dirs, q)}
    for d in range(1, 19):
        assert int(node[list(dirs).index(d)]) == s - (L.E[d, 0] + 6 * (L.E[d, 1] + 6 * L.E[d, 2]))
    # e_2 = (-1,0,0): b = (3,3,2), b - L = (0.8,-0.1,0.1): sqrt(0.66)
    assert abs(got[2] - math.sqrt(0.66)) < 1e-7
    # e_5 = (0,0,1): b = (2,3,1), b - L = (-0.2,-0.1,-0.9): sqrt(0.86)
    assert abs(got[5] - math.sqrt(0.86)) < 1e-7
    # e_6 = (0,0,-1): b = (2,3,3), b - L = (-0.2,-0.1,1.1): sqrt(1.26) > 1, clipped
    assert got[6] == 1.0
    # e_12 = (-1,-1,0): b = (3,4,2), b - L = (0.8,0.9,0.1): sqrt(1.46)/sqrt(2)
    assert abs(got[12] - math.sqrt(1.46) / SQ2) < 1e-7
    # e_1 = (1,0,0): b = (1,3,2), b - L = (-1.2,-0.1,0.1): sqrt(1.46) > 1, clipped
    assert got[1] == 1.0


def _brute(verts, tris, shape, periodic, tag_in):
    """The rule restated with plain loops over nodes, directions and markers."""
    nx, ny, nz = shape
    dims = shape
    tag = [int(t) for t in tag_in]
    cells = []
    for a, b, c in tris:
        Lm = [(verts[a][k] + verts[b][k] + verts[c][k]) / 3.0 for k in range(3)]
        raw = [math.floor(Lm[k] + 0.5) for k in range(3)]
        cell = []
        ok = True
        for k in range(3):
            if periodic[k]:
                cell.append(raw[k] % dims[k])
            elif 0 <= raw[k] < dims[k]:
                cell.append(raw[k])
            else:
                ok = False
        if ok:
            flat = cell[0] + nx * (cell[1] + ny * cell[2])
            tag[flat] = 1
            cells.append((flat, raw, Lm))
    links = []
    for n in range(nx * ny * nz):
        if tag[n]:
            continue
        p = (n % nx, (n // nx) % ny, n // (nx * ny))
        for i in range(1, 19):
            e = L.E[i]
            sc = []
            ok = True
            for k in range(3):
                v = p[k] + int(e[k])
                if periodic[k]:
                    v %= dims[k]
                elif not 0 <= v < dims[k]:
                    ok = False
                sc.append(v)
            if not ok:
                continue
            sflat = sc[0] + nx * (sc[1] + ny * sc[2])
            if not tag[sflat]:
                continue
            best = math.inf
            for flat, raw, Lm in cells:
                if flat != sflat:
                    continue
                # x_b seen from this marker: its raw cell minus e_i (unwrapped)
                xb = [raw[k] - int(e[k]) for k in range(3)]
                dx, dy, dz = xb[0] - Lm[0], xb[1] - Lm[1], xb[2] - Lm[2]
                best = min(best, math.sqrt((dx * dx + dy * dy) + dz * dz))
            elen = 1.0 if i <= 6 else SQ2
            qv = 0.5 if best == math.inf else best / elen
            links.append((n, i, np.float32(min(max(qv, 1e-6), 1.0))))
    return np.array(tag, np.uint8), links


def test_brute_force_on_tiny_inputs():
    rng = np.random.default_rng(7)
    for shape, periodic in (((7, 6, 5), (False, False, False)), ((6, 7, 5), (True, False, True)),
                            ((5, 5, 6), (True, True, True))):
        nv, nt = 30, 24
        V = rng.uniform(-1.0, max(shape) + 0.5, size=(nv, 3))
        T = rng.integers(0, nv, size=(nt, 3))
        tag_in = (rng.uniform(size=shape[0] * shape[1] * shape[2]) < 0.05).astype(np.uint8)
        tag, node, dirs, q = Wl.voxelise_markers(V, T, shape, periodic, tag_in)
        tb, lb = _brute(V.tolist(), T.tolist(), shape, periodic, tag_in)
        assert np.array_equal(tag, tb)
        assert len(lb) == len(node)
        for (n, i, qq), a, b, c in zip(lb, node, dirs, q):
            assert (n, i) == (int(a), int(b))
            assert qq == c
        assert (q >= 1e-6).all() and (q <= 1.0).all()


def _tube_flow(R, nx=4, tau=0.8, h=0.3):
    n = int(2 * R + 6)
    c = (n - 1) / 2.0
    V, T = Ms.tube_mesh(-0.5, nx - 0.5, R, c, c, h, periodic_x=True)
    idx = np.arange(nx * n * n)
    Y, Z = (idx // nx) % n, idx // (nx * n)
    r = np.hypot(Y - c, Z - c)
    tag, node, dirs, q = Wl.voxelise_markers(V, T, (nx, n, n), (True, False, False),
                                             (r > R + 1.5).astype(np.uint8))
    links = np.zeros(len(node), dtype=G.LINK_DTYPE)
    links["node"], links["dir"], links["q"] = node, dirs, q
    g = 1e-6
    lat = L.Lattice(nx, n, n, tau, tag, links, [G.Face() for _ in range(6)], (True, False, False),
                    body_force=np.array([g, 0.0, 0.0]))
    nu = L.viscosity(tau)
    uex = np.where(r < R, g / (4.0 * nu) * (R * R - r * r), 0.0)
    f = lat.init_equilibrium(None, np.stack([uex, 0 * uex, 0 * uex], axis=1) * lat.fluid[:, None])
    for _ in range(int(3 * R * R / nu)):
        f = lat.step(f)
    _, u = lat.macroscopic(f)
    inside = lat.fluid & (r < R - 0.5)
    err = np.linalg.norm(u[inside, 0] - uex[inside]) / np.linalg.norm(uex[inside])
    centre = u[lat.fluid & (r == r.min()), 0].mean() / (g * R * R / (4.0 * nu))
    return err, centre


def test_tube_flow_with_marker_walls():
    """Hagen-Poiseuille in a periodic tube whose wall is only a triangulation
    (edges 0.3 lu): the marker rule is first order in the wall position (a
    solid cell is any cell the surface touches, and q >= 1/2), so the flow
    is slower than the closed form by an amount that shrinks with the
    radius: centreline 0.79 (R = 4) and 0.88 (R = 6) of g R^2 / 4 nu, the
    relative L2 error falling from 0.25 to 0.17."""
    e4, c4 = _tube_flow(4.0)
    e6, c6 = _tube_flow(6.0)
    assert 0.75 < c4 < c6 < 1.0, (c4, c6)
    assert e6 < e4 < 0.3, (e4, e6)
