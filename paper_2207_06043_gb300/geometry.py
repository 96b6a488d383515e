"""Seeded, synthetic lattice geometries: the input side of the solver.

This module builds what the library's ``ibl_set_geometry`` / face calls take:
a per-node fluid/solid tag, the list of wall links with their
Bouzidi-Firdaouss-Lallemand distance q (Eq. qbouzidi, measured here to the
analytic wall instead of to wall markers), and the Dirichlet data of the six
box faces (a Poiseuille inlet with peak u_max, pressure outlets; Section
"Computational set-up and boundary conditions").  It holds no lattice
Boltzmann, immersed-boundary or membrane arithmetic: it is shared by the CPU
oracle and the CUDA path only as a producer of inputs.

Conventions
-----------
* node index = x + nx*(y + ny*z); arrays are flat, x fastest.
* tag: 0 = fluid, 1 = solid.
* direction numbering is the one of Eq. e_i (19 columns, e_0 = 0).
* a wall link (node, i, q) says that node + e_i is solid and that the wall
  crosses the link at fraction q of its length, measured from ``node``.
* faces: 0 = x-, 1 = x+, 2 = y-, 3 = y+, 4 = z-, 5 = z+.  A face array is
  laid out with the lower remaining axis fastest (face 0/1: y + ny*z; face 2/3:
  x + nx*z; face 4/5: x + nx*y).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Sequence

import numpy as np

# Velocity set of Eq. e_i, used here only to enumerate wall links.
E19 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0],
    [0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, -1],
], dtype=np.int64).T

FLUID = 0
SOLID = 1

FACE_NONE = 0
FACE_VELOCITY = 1
FACE_PRESSURE = 2

LINK_DTYPE = np.dtype([("node", "<u4"), ("dir", "<u4"), ("q", "<f4"), ("dq", "<f4")])


@dataclasses.dataclass
class Face:
    kind: int = FACE_NONE           # FACE_NONE / FACE_VELOCITY / FACE_PRESSURE
    rho: float = 1.0                # prescribed density of a pressure face
    velocity: Optional[np.ndarray] = None  # (n_face, 3) float32 of a velocity face


@dataclasses.dataclass
class Geometry:
    nx: int
    ny: int
    nz: int
    periodic: tuple
    tag: np.ndarray                 # (N,) uint8
    links: np.ndarray               # (L,) LINK_DTYPE
    faces: List[Face]
    sdf: Optional[Callable] = None  # signed distance, < 0 in the fluid
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_fluid(self) -> int:
        return int(np.count_nonzero(self.tag == FLUID))

    def coords(self):
        n = np.arange(self.n_nodes, dtype=np.int64)
        return n % self.nx, (n // self.nx) % self.ny, n // (self.nx * self.ny)


def face_shape(face: int, nx: int, ny: int, nz: int):
    """Number of nodes along the two in-face axes (fast, slow)."""
    return {0: (ny, nz), 1: (ny, nz), 2: (nx, nz), 3: (nx, nz), 4: (nx, ny), 5: (nx, ny)}[face]


# ----------------------------------------------------------------------------
# signed distance functions (negative inside the fluid)
# ----------------------------------------------------------------------------

def box_duct_sdf(p0, p1, half_width, half_height=None):
    """Square-section duct whose axis runs from p0 to p1 in the x-y plane.

    The cross-section is 2*half_width wide (in the x-y plane, normal to the axis)
    and 2*half_height tall (along z).  Exact box distance."""
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    hh = half_width if half_height is None else half_height
    axis = p1 - p0
    length = float(np.linalg.norm(axis))
    a = axis / length
    b = np.array([-a[1], a[0], 0.0])
    c = np.array([0.0, 0.0, 1.0])
    centre = 0.5 * (p0 + p1)

    def f(P):
        dx = P[:, 0] - centre[0]
        dy = P[:, 1] - centre[1]
        dz = P[:, 2] - centre[2]
        s = np.abs(dx * a[0] + dy * a[1]) - 0.5 * length
        t = np.abs(dx * b[0] + dy * b[1]) - half_width
        w = np.abs(dz) - hh
        so, to, wo = np.maximum(s, 0.0), np.maximum(t, 0.0), np.maximum(w, 0.0)
        outside = np.sqrt(so * so + to * to + wo * wo)
        inside = np.minimum(np.maximum(np.maximum(s, t), w), 0.0)
        return outside + inside
    return f


def slab_sdf(normal, offset, half_width, period=None):
    """Planar channel |n.x - offset| < half_width, optionally repeated with a
    perpendicular period (used for inclined periodic channels)."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)

    def f(P):
        s = P @ n - offset
        if period is not None:
            s = (s + 0.5 * period) % period - 0.5 * period
        return np.abs(s) - half_width
    return f


def round_union(d1, d2, r):
    """Union of two fluid regions whose concave corners are filled with a
    circular fillet of radius r (r = 0: plain union)."""
    if r <= 0:
        return np.minimum(d1, d2)
    u = np.maximum(r - d1, 0.0)
    v = np.maximum(r - d2, 0.0)
    return np.maximum(r, np.minimum(d1, d2)) - np.sqrt(u * u + v * v)


# ----------------------------------------------------------------------------
# voxelisation, links, faces
# ----------------------------------------------------------------------------

def _node_positions(nx, ny, nz):
    n = np.arange(nx * ny * nz, dtype=np.int64)
    return np.stack([n % nx, (n // nx) % ny, n // (nx * ny)], axis=-1).astype(np.float64)


def _bisect_root(sdf, a, b, iters=40):
    """Root of sdf on the segments a->b (sdf(a) < 0 <= sdf(b)); returns the
    fraction along the segment."""
    lo = np.zeros(a.shape[0])
    hi = np.ones(a.shape[0])
    d = b - a
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        val = sdf(a + mid[:, None] * d)
        inside = val < 0.0
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return 0.5 * (lo + hi)


def voxelise(sdf, nx, ny, nz, periodic=(False, False, False), sdf_param=None,
             q_min=1e-6):
    """Tag nodes (fluid where sdf < 0) and build the wall links.

    Nodes on an edge or corner of the box (on two or more non-periodic faces)
    are tagged solid so that every fluid face node lies on exactly one face.
    A link toward such a forced-solid node (no sign change of the SDF) gets
    q = 1/2 (halfway bounce-back)."""
    P = _node_positions(nx, ny, nz)
    d = sdf(P)
    tag = np.where(d < 0.0, FLUID, SOLID).astype(np.uint8)
    dims = (nx, ny, nz)
    on_face = np.zeros(P.shape[0], dtype=np.int64)
    for ax in range(3):
        if not periodic[ax]:
            c = P[:, ax]
            on_face += (c == 0) | (c == dims[ax] - 1)
    tag[on_face >= 2] = SOLID

    fluid = np.nonzero(tag == FLUID)[0]
    X = fluid % nx
    Y = (fluid // nx) % ny
    Z = fluid // (nx * ny)
    nodes, dirs = [], []
    for i in range(1, 19):
        ex, ey, ez = E19[i]
        sx, sy, sz = X + ex, Y + ey, Z + ez
        ok = np.ones(fluid.shape[0], dtype=bool)
        for ax, (s, n) in enumerate(((sx, nx), (sy, ny), (sz, nz))):
            if periodic[ax]:
                s %= n
            else:
                ok &= (s >= 0) & (s < n)
        nb = np.where(ok, sx + nx * (sy + ny * sz), 0)
        hit = ok & (tag[nb] == SOLID)
        nodes.append(fluid[hit])
        dirs.append(np.full(int(hit.sum()), i, dtype=np.int64))
    nodes = np.concatenate(nodes) if nodes else np.zeros(0, np.int64)
    dirs = np.concatenate(dirs) if dirs else np.zeros(0, np.int64)
    order = np.lexsort((dirs, nodes))
    nodes, dirs = nodes[order], dirs[order]

    a = P[nodes]
    b = a + E19[dirs].astype(np.float64)
    q = np.full(nodes.shape[0], 0.5)
    dq = np.zeros(nodes.shape[0])
    if nodes.shape[0]:
        sb = sdf(b)
        real = sb >= 0.0   # the SDF changes sign along the link
        if real.any():
            q[real] = _bisect_root(sdf, a[real], b[real])
            if sdf_param is not None:
                # dq/d(param) by a central difference of the root position
                h = 1e-4
                fp = sdf_param(+h)
                fm = sdf_param(-h)
                ar, br = a[real], b[real]
                ok = (fp(ar) < 0) & (fp(br) >= 0) & (fm(ar) < 0) & (fm(br) >= 0)
                qp = _bisect_root(fp, ar, br)
                qm = _bisect_root(fm, ar, br)
                dq_r = np.where(ok, (qp - qm) / (2 * h), 0.0)
                dq[real] = dq_r
    q = np.clip(q, q_min, 1.0)
    links = np.zeros(nodes.shape[0], dtype=LINK_DTYPE)
    links["node"] = nodes.astype(np.uint32)
    links["dir"] = dirs.astype(np.uint32)
    links["q"] = q.astype(np.float32)
    links["dq"] = dq.astype(np.float32)
    return tag, links


def face_node_mask(geom_tag, nx, ny, nz, face):
    """Boolean (n_face,) mask of fluid nodes on a face, in face layout."""
    t = geom_tag.reshape(nz, ny, nx)
    sl = {0: t[:, :, 0], 1: t[:, :, nx - 1], 2: t[:, 0, :], 3: t[:, ny - 1, :],
          4: t[0, :, :], 5: t[nz - 1, :, :]}[face]
    return (sl == FLUID).reshape(-1)


def duct_poiseuille(yy, zz, half_a, half_b, u_max, n_terms=41):
    """Fully developed laminar velocity in a rectangular duct |y|<a, |z|<b
    (Fourier series solution of the Poisson problem), scaled to peak u_max."""
    def series(y, z):
        s = np.zeros_like(y, dtype=np.float64)
        for k in range(n_terms):
            n = 2 * k + 1
            beta = n * math.pi / (2 * half_a)
            s += ((-1) ** k / n ** 3) * (1.0 - np.cosh(beta * z) / np.cosh(beta * half_b)) * np.cos(beta * y)
        return s
    peak = series(np.zeros(1), np.zeros(1))[0]
    u = u_max * series(yy, zz) / peak
    inside = (np.abs(yy) < half_a) & (np.abs(zz) < half_b)
    return np.where(inside, u, 0.0)


def inlet_x_minus(tag, nx, ny, nz, yc, zc, half, u_max):
    """Velocity data of face 0 (x = 0): square-duct Poiseuille along +x."""
    Y, Z = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nz, dtype=np.float64), indexing="xy")
    u = duct_poiseuille(Y.reshape(-1) - yc, Z.reshape(-1) - zc, half, half, u_max)
    mask = face_node_mask(tag, nx, ny, nz, 0)
    vel = np.zeros((ny * nz, 3), dtype=np.float32)
    vel[:, 0] = np.where(mask, u, 0.0).astype(np.float32)
    return vel


def _faces_for_duct_flow(tag, nx, ny, nz, periodic, yc, zc, half, u_max, rho_out=1.0):
    faces = [Face() for _ in range(6)]
    if not periodic[0]:
        faces[0] = Face(FACE_VELOCITY, 1.0, inlet_x_minus(tag, nx, ny, nz, yc, zc, half, u_max))
    for f in range(1, 6):
        ax = f // 2
        if periodic[ax]:
            continue
        if face_node_mask(tag, nx, ny, nz, f).any():
            faces[f] = Face(FACE_PRESSURE, rho_out, None)
    return faces


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def straight_duct(nx, ny, nz, D, u_max=0.02, periodic_x=False, rho_out=1.0,
                  centre=None):
    """Square duct of side D along x, centred in (y, z).  With periodic_x the
    ends wrap (drive it with a body force); otherwise x=0 is a Poiseuille
    velocity inlet and x=nx-1 a pressure outlet."""
    yc = (ny - 1) / 2 if centre is None else centre[0]
    zc = (nz - 1) / 2 if centre is None else centre[1]
    h = D / 2.0
    sdf = box_duct_sdf((-4.0 * nx, yc, zc), (5.0 * nx, yc, zc), h)
    periodic = (bool(periodic_x), False, False)
    tag, links = voxelise(sdf, nx, ny, nz, periodic)
    faces = _faces_for_duct_flow(tag, nx, ny, nz, periodic, yc, zc, h, u_max, rho_out)
    return Geometry(nx, ny, nz, periodic, tag, links, faces, sdf,
                    dict(kind="straight_duct", D=D, u_max=u_max, yc=yc, zc=zc))


def periodic_box(nx, ny, nz):
    tag = np.zeros(nx * ny * nz, dtype=np.uint8)
    links = np.zeros(0, dtype=LINK_DTYPE)
    return Geometry(nx, ny, nz, (True, True, True), tag, links, [Face() for _ in range(6)], None,
                    dict(kind="periodic_box"))


def inclined_channel(width, slope_num=1, slope_den=2, ly=None, offset=0.37):
    """Planar channel of perpendicular width ``width`` whose axis has slope
    slope_num/slope_den in the x-y plane, periodic in x and y (box lx = ly *
    slope_den / slope_num so that the stripes tile) and one node thick in z."""
    ang = math.atan2(slope_num, slope_den)
    n = np.array([-math.sin(ang), math.cos(ang), 0.0])
    if ly is None:
        # perpendicular period must exceed the width plus a few wall nodes
        ly = int(math.ceil((width + 4.0) / math.cos(ang))) + 1
        while (ly * slope_den) % slope_num:
            ly += 1
    lx = ly * slope_den // slope_num
    period = ly * math.cos(ang)
    centre = 0.5 * ly * math.cos(ang) + offset
    sdf = slab_sdf(n, centre, width / 2.0, period)
    periodic = (True, True, True)
    tag, links = voxelise(sdf, lx, ly, 1, periodic)
    return Geometry(lx, ly, 1, periodic, tag, links, [Face() for _ in range(6)], sdf,
                    dict(kind="inclined_channel", width=width, normal=n, centre=centre,
                         period=period, axis=np.array([math.cos(ang), math.sin(ang), 0.0])))


def _bifurcation_sdf(nx, ny, nz, D, half_angle_deg, r_j, x_junction, daughter_ratio,
                     levels=1, centre=None):
    yc = (ny - 1) / 2 if centre is None else centre[0]
    zc = (nz - 1) / 2 if centre is None else centre[1]
    far = 4.0 * (nx + ny + nz)
    th = math.radians(half_angle_deg)
    h0 = D / 2.0
    main = box_duct_sdf((-far, yc, zc), (x_junction, yc, zc), h0, h0)

    # tree of segments: each entry (start point, direction angle, half width, level)
    parts = [main]
    pieces = [(np.array([x_junction, yc, zc]), 0.0, h0, 0)]
    segs = []
    while pieces:
        p, ang, hw, lev = pieces.pop()
        hd = hw * daughter_ratio
        for sgn in (+1.0, -1.0):
            a = ang + sgn * th
            direc = np.array([math.cos(a), math.sin(a), 0.0])
            start = p - hw * np.array([math.cos(ang), math.sin(ang), 0.0])
            if lev + 1 < levels:
                seg_len = 1.5 * (2 * hd)
                end = p + seg_len * direc
                segs.append((start, end, hd))
                pieces.append((end, a, hd, lev + 1))
            else:
                segs.append((start, start + far * direc, hd))
    duct_sdfs = [box_duct_sdf(s, e, hd, min(hd, h0)) for (s, e, hd) in segs]

    def sdf(P, rj=r_j):
        d = main(P)
        for f in duct_sdfs:
            d = round_union(d, f(P), rj)
        return d
    return sdf, yc, zc, h0


def bifurcation(nx, ny, nz, D, half_angle_deg=45.0, r_j=0.0, u_max=0.02, x_junction=None,
                daughter_ratio=1.0 / math.sqrt(2.0), levels=1, rho_out=1.0, with_dq=False):
    """Symmetric square-duct bifurcation: a main duct of side D along +x from the
    inlet (x=0) to the junction at x_junction, splitting into two daughters of
    side daughter_ratio*D at +-half_angle in the x-y plane (levels=2 splits each
    daughter once more).  The junction's concave corners are rounded by a
    fillet of radius r_j (0 = sharp).  Daughters leave through the box faces,
    which are pressure outlets."""
    if x_junction is None:
        x_junction = 0.4 * nx
    sdf, yc, zc, h0 = _bifurcation_sdf(nx, ny, nz, D, half_angle_deg, r_j, x_junction,
                                        daughter_ratio, levels)
    sdf_param = None
    if with_dq:
        def sdf_param(dr):
            return lambda P: sdf(P, r_j + dr)
    periodic = (False, False, False)
    tag, links = voxelise(sdf, nx, ny, nz, periodic, sdf_param=sdf_param)
    faces = _faces_for_duct_flow(tag, nx, ny, nz, periodic, yc, zc, h0, u_max, rho_out)
    return Geometry(nx, ny, nz, periodic, tag, links, faces, sdf,
                    dict(kind="bifurcation", D=D, half_angle=half_angle_deg, r_j=r_j,
                         u_max=u_max, x_junction=x_junction, yc=yc, zc=zc, levels=levels))


def cylinder_sdf(p0, p1, radius):
    """Circular-section duct whose axis runs from p0 to p1 (flat ends).  Exact
    distance of a finite cylinder."""
    p0 = np.asarray(p0, dtype=np.float64)
    p1 = np.asarray(p1, dtype=np.float64)
    axis = p1 - p0
    length = float(np.linalg.norm(axis))
    a = axis / length
    centre = 0.5 * (p0 + p1)

    def f(P):
        r = P - centre[None, :]
        s = r @ a
        radial = np.sqrt(np.maximum((r * r).sum(axis=1) - s * s, 0.0)) - radius
        axial = np.abs(s) - 0.5 * length
        ro, ao = np.maximum(radial, 0.0), np.maximum(axial, 0.0)
        return np.sqrt(ro * ro + ao * ao) + np.minimum(np.maximum(radial, axial), 0.0)
    return f


def circular_bifurcation(d=30.0, half_angle_deg=30.0, smooth=False, u_max=0.003, main_len=6.7, branch_len=5.0,
                         daughter_ratio=0.7, flat_width=None, margin=3, rho_out=1.0):
    """The paper's bifurcation (Section "Computational set-up and boundary
    conditions"): a circular main duct of diameter d along +x, main_len * d
    long, splitting into two circular daughters of diameter daughter_ratio * d
    and branch_len * d long at +-half_angle in the x-y plane.  smooth=False
    joins the three ducts as they are (a sharp cusp between the daughters);
    smooth=True also fills the tip of the solid cusp, up to where it is
    flat_width wide (default d / 3), leaving a flat wall across the flow that
    faces the main duct: the flat-topped junction.  The box encloses the ducts with `margin` solid
    nodes; the inlet (x = 0) carries the circular Poiseuille profile of peak
    u_max and every daughter end face is a pressure outlet."""
    th = math.radians(half_angle_deg)
    R, r = d / 2.0, daughter_ratio * d / 2.0
    L0, L1 = main_len * d, branch_len * d
    span_y = 2.0 * (L1 * math.sin(th) + r * math.cos(th)) + 2.0 * margin
    ny = int(math.ceil(max(d + 2 * margin, span_y))) + 1
    nz = int(math.ceil(d)) + 2 * margin + 1
    yc, zc = (ny - 1) / 2.0, (nz - 1) / 2.0
    xj = L0
    nx = int(math.ceil(xj + L1 * math.cos(th) + r * math.sin(th))) + 1
    far = 2.0 * d
    main = cylinder_sdf((-far, yc, zc), (xj, yc, zc), R)
    ducts = []
    for sgn in (1.0, -1.0):
        direc = np.array([math.cos(th), sgn * math.sin(th), 0.0])
        start = np.array([xj, yc, zc]) - R * np.array([1.0, 0.0, 0.0])
        ducts.append(cylinder_sdf(start, start + (L1 + far) * direc, r))
    # the inner walls of the two daughters (parallel to their axes, which
    # start on the main axis at xj - R) meet on the main axis at the cusp; the
    # solid cusp between them is |y - yc| < (x - x_cusp) tan th
    x_cusp = xj - R + r / math.sin(th)
    if flat_width is None:
        flat_width = d / 3.0
    x_cut = x_cusp + 0.5 * flat_width / math.tan(th)

    def wedge(P):
        # the solid cusp from its tip to x_cut, within the daughters' height
        lateral = np.abs(P[:, 1] - yc) - (P[:, 0] - x_cusp) * math.tan(th)
        return np.maximum.reduce([lateral * math.cos(th), P[:, 0] - x_cut, (x_cusp - 1.0) - P[:, 0],
                                  np.abs(P[:, 2] - zc) - r])

    def sdf(Pts):
        dd = main(Pts)
        for f in ducts:
            dd = np.minimum(dd, f(Pts))
        if smooth:
            dd = np.minimum(dd, wedge(Pts))
        return dd

    periodic = (False, False, False)
    tag, links = voxelise(sdf, nx, ny, nz, periodic)
    faces = [Face() for _ in range(6)]
    Y, Z = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nz, dtype=np.float64), indexing="xy")
    rr2 = ((Y.reshape(-1) - yc) ** 2 + (Z.reshape(-1) - zc) ** 2) / (R * R)
    mask = face_node_mask(tag, nx, ny, nz, 0)
    vel = np.zeros((ny * nz, 3), dtype=np.float32)
    vel[:, 0] = np.where(mask & (rr2 < 1.0), u_max * (1.0 - rr2), 0.0).astype(np.float32)
    faces[0] = Face(FACE_VELOCITY, 1.0, vel)
    for f in range(1, 6):
        if face_node_mask(tag, nx, ny, nz, f).any():
            faces[f] = Face(FACE_PRESSURE, rho_out, None)
    return Geometry(nx, ny, nz, periodic, tag, links, faces, sdf,
                    dict(kind="circular_bifurcation", D=d, half_angle=half_angle_deg, smooth=bool(smooth),
                         u_max=u_max, x_junction=xj, x_cusp=x_cusp, x_cut=x_cut if smooth else None,
                         yc=yc, zc=zc))


def crop_x(geom: Geometry, x1: int) -> Geometry:
    """The slab 0 <= x < x1 of a geometry whose x axis is not periodic: wall
    links that leave the slab are dropped and the fluid nodes of the cut plane
    become a pressure face (density 1)."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    t3 = geom.tag.reshape(nz, ny, nx)[:, :, :x1]
    tag = np.ascontiguousarray(t3).reshape(-1).copy()
    # nodes of the cut plane that also lie on another face become solid
    X = np.arange(tag.size) % x1
    Y = (np.arange(tag.size) // x1) % ny
    Z = np.arange(tag.size) // (x1 * ny)
    edge = (X == x1 - 1) & ((Y == 0) | (Y == ny - 1) | (Z == 0) | (Z == nz - 1))
    tag[edge] = SOLID
    lx = geom.links["node"] % nx
    ly = (geom.links["node"] // nx) % ny
    lz = geom.links["node"] // (nx * ny)
    tx = lx + E19[geom.links["dir"].astype(np.int64), 0]
    keep = (lx < x1) & (tx < x1) & (tx >= 0)
    links = geom.links[keep].copy()
    links["node"] = (lx[keep] + x1 * (ly[keep] + ny * lz[keep])).astype(np.uint32)
    # drop links that start at nodes made solid above
    links = links[tag[links["node"]] == FLUID]
    faces = [Face(f.kind, f.rho, f.velocity) for f in geom.faces]
    if faces[0].kind == FACE_VELOCITY:
        faces[0] = Face(FACE_VELOCITY, 1.0, faces[0].velocity)
    for f in (2, 3, 4, 5):
        if faces[f].kind == FACE_VELOCITY:
            raise ValueError("crop_x keeps only x- velocity faces")
        faces[f] = Face(FACE_PRESSURE, 1.0, None) if face_node_mask(tag, x1, ny, nz, f).any() else Face()
    faces[1] = Face(FACE_PRESSURE, 1.0, None)
    info = dict(geom.info)
    info["cropped_from"] = (nx, ny, nz)
    return Geometry(x1, ny, nz, geom.periodic, tag, links, faces, None, info)
