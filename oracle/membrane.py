"""FP64 membrane mechanics and capsule diagnostics (Section "Immersed-Structure
Transport"): mesh topology, stretching, bending and volume forces, the
hydrodynamic pressure/viscous forces from probes, inter-body repulsion, and
the volume / area / centroid / Taylor-deformation reductions.

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.
"""
from __future__ import annotations

import math

import numpy as np

from . import ib
from .lattice import viscosity


# The functions below also run on complex arrays for complex-step derivative
# checks, d g(x)/dx . v = Im g(x + i h v) / h: norms are written as the
# analytic sqrt(sum x^2), and the angle and eigenvalue helpers carry the
# first-order complex part; every discrete decision looks at real parts.
def _norm(v, axis=-1):
    return np.sqrt((v * v).sum(axis=axis))


def _atan2(s, c):
    """arctan2 with the complex-step derivative (c ds - s dc)/(s^2 + c^2)."""
    if not (np.iscomplexobj(s) or np.iscomplexobj(c)):
        return np.arctan2(s, c)
    sr, cr = np.real(s), np.real(c)
    return np.arctan2(sr, cr) + 1j * (cr * np.imag(s) - sr * np.imag(c)) / (sr * sr + cr * cr)


def _eigvalsh(C):
    """Ascending eigenvalues of a symmetric 3x3 matrix, with the first-order
    complex part v_i^T Im(C) v_i of each (distinct) eigenvalue."""
    if not np.iscomplexobj(C):
        return np.linalg.eigvalsh(C)
    w, V = np.linalg.eigh(np.real(C))
    return w + 1j * np.einsum("ji,jk,ki->i", V, np.imag(C), V)


class Topology:
    """Edges and hinges of a closed triangle mesh with outward CCW triangles.

    For every undirected edge {p, q} (p < q): tri_a holds the directed edge
    p->q and has wing vertex v1, tri_b holds q->p and has wing v4; the hinge is
    (v1, v2=p, v3=q, v4) so that tri_a = (v1, v2, v3) and tri_b = (v4, v3, v2)."""

    def __init__(self, tris):
        tris = np.asarray(tris, dtype=np.int64)
        self.tris = tris
        self.nv = int(tris.max()) + 1
        half = {}
        for t, (a, b, c) in enumerate(tris):
            for (u, v, w) in ((a, b, c), (b, c, a), (c, a, b)):
                half[(u, v)] = (t, w)
        hinges = []
        for (u, v), (t, w) in half.items():
            if u < v:
                t2, w2 = half[(v, u)]
                hinges.append((w, u, v, w2, t, t2))
        h = np.array(sorted(hinges, key=lambda r: (r[1], r[2])), dtype=np.int64)
        self.hinge = h[:, :4]
        self.edge = h[:, 1:3]
        self.edge_tris = h[:, 4:6]


def triangle_vectors(X, tris):
    """Per-triangle cross product N = (b-a) x (c-a) (twice the area, outward)."""
    a, b, c = X[tris[:, 0]], X[tris[:, 1]], X[tris[:, 2]]
    return np.cross(b - a, c - a)


def vertex_areas_normals(X, tris, nv):
    """Reading M1: A_v = (1/3) sum of the adjacent triangle areas; n_v = the
    normalised area-weighted sum of the adjacent triangle normals."""
    N = triangle_vectors(X, tris)
    area = 0.5 * _norm(N, axis=1)
    Av = np.zeros(nv, dtype=N.dtype)
    nv_acc = np.zeros((nv, 3), dtype=N.dtype)
    for j in range(3):
        np.add.at(Av, tris[:, j], area / 3.0)
        np.add.at(nv_acc, tris[:, j], 0.5 * N)
    nrm = nv_acc / _norm(nv_acc, axis=1)[:, None]
    return Av, nrm


def dihedral_angles(X, hinge):
    """Signed angle between the outward normals of the two triangles of each
    hinge (positive where the surface is convex)."""
    v1, v2, v3, v4 = (X[hinge[:, j]] for j in range(4))
    nA = np.cross(v2 - v1, v3 - v1)
    nB = np.cross(v3 - v4, v2 - v4)
    e = v3 - v2
    e_hat = e / _norm(e, axis=1)[:, None]
    s = np.einsum("ij,ij->i", np.cross(nA, nB), e_hat)
    c = np.einsum("ij,ij->i", nA, nB)
    return _atan2(s, c)


def dihedral_gradients(X, hinge):
    """d theta / d v1..v4 for each hinge (4, H, 3): the standard hinge-angle
    gradient (wing vertices move along their triangle normal with lever arm
    height = 2 area / |e|; edge vertices by translation/rotation invariance)."""
    v1, v2, v3, v4 = (X[hinge[:, j]] for j in range(4))
    nA = np.cross(v2 - v1, v3 - v1)
    nB = np.cross(v3 - v4, v2 - v4)
    e = v3 - v2
    L = _norm(e, axis=1)
    e_hat = e / L[:, None]
    a2 = np.einsum("ij,ij->i", nA, nA)
    b2 = np.einsum("ij,ij->i", nB, nB)
    gA = nA / a2[:, None]
    gB = nB / b2[:, None]
    u1 = L[:, None] * gA
    u4 = L[:, None] * gB
    u2 = (np.einsum("ij,ij->i", v1 - v3, e_hat)[:, None] * gA
          + np.einsum("ij,ij->i", v4 - v3, e_hat)[:, None] * gB)
    u3 = -(np.einsum("ij,ij->i", v1 - v2, e_hat)[:, None] * gA
           + np.einsum("ij,ij->i", v4 - v2, e_hat)[:, None] * gB)
    return -np.stack([u1, u2, u3, u4])


class CapsuleRest:
    """Rest quantities of one capsule (computed once from the initial mesh)."""

    def __init__(self, X0, tris, params, tau):
        self.topo = Topology(tris)
        X0 = np.asarray(X0, dtype=np.float64)
        t = self.topo
        self.l0 = _norm(X0[t.edge[:, 1]] - X0[t.edge[:, 0]], axis=1)
        tri_area = 0.5 * _norm(triangle_vectors(X0, t.tris), axis=1)
        self.theta0 = dihedral_angles(X0, t.hinge)
        d = diagnostics(X0, t.tris)
        self.V0 = d["volume"]
        self.S0 = d["area"]
        self.radius = (3.0 * self.V0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        nu = viscosity(tau)
        rho_f = 1.0
        self.rigid = bool(params.get("rigid", 0))
        Ca = params.get("Ca", 0.01)
        u_ref = params.get("u_ref", 0.02)
        # Ca = rho nu u_ref / k_s0  (Section "Deforming bodies constitutive model")
        self.ks0 = rho_f * nu * u_ref / Ca if np.real(Ca) > 0 else 0.0
        # Reading S-a: k_s,l = k_s0 T (A_a + A_b) / l0^2 with T = 1
        self.ks = self.ks0 * (tri_area[t.edge_tris[:, 0]] + tri_area[t.edge_tris[:, 1]]) / self.l0 ** 2
        # Eb = k_b / (k_s,l r^2)  ->  k_b = Eb k_s,l r^2 (per hinge = per edge)
        self.kb = params.get("Eb", 0.001) * self.ks * self.radius ** 2
        self.kv = params.get("kv", 1.0)
        self.density_ratio = params.get("density_ratio", 1.1)
        self.mass = self.density_ratio * rho_f * self.V0
        self.mv = self.mass / t.nv


def stretch_energy(X, rest):
    """Eq. strainPot summed over edges."""
    e = rest.topo.edge
    l = _norm(X[e[:, 0]] - X[e[:, 1]], axis=1)
    return 0.5 * np.sum(rest.ks * (l - rest.l0) ** 2)


def stretch_forces(X, rest):
    """Eq. strainFor: F_1 = -k_s,l (l - l0) r_12 / l, F_2 = -F_1, per edge."""
    e = rest.topo.edge
    r12 = X[e[:, 0]] - X[e[:, 1]]
    l = _norm(r12, axis=1)
    F1 = -(rest.ks * (l - rest.l0) / l)[:, None] * r12
    out = np.zeros(X.shape, dtype=F1.dtype)
    np.add.at(out, e[:, 0], F1)
    np.add.at(out, e[:, 1], -F1)
    return out


def bending_energy(X, rest):
    """Reading S-b: V = k_b [1 - cos(theta - theta0)] per hinge, the potential
    whose gradient has the beta_b = k_b sin(theta - theta0)/sin(theta) factor of
    Eq. bendFor."""
    th = dihedral_angles(X, rest.topo.hinge)
    return np.sum(rest.kb * (1.0 - np.cos(th - rest.theta0)))


def bending_forces(X, rest):
    """F = -dV/dx = -k_b sin(theta - theta0) d theta/dx on the 4 hinge nodes."""
    h = rest.topo.hinge
    th = dihedral_angles(X, h)
    g = dihedral_gradients(X, h)                  # (4,H,3)
    coef = -(rest.kb * np.sin(th - rest.theta0))   # (H,)
    out = np.zeros(X.shape, dtype=np.result_type(coef, g))
    for j in range(4):
        np.add.at(out, h[:, j], coef[:, None] * g[j])
    return out


def volume_forces(X, rest, V, Av, nrm):
    """Eq. volFor with the restoring sign (Reading S-c):
    F_i = k_v (1 - V/V0) n_i A_i, n outward."""
    return (rest.kv * (1.0 - V / rest.V0) * Av)[:, None] * nrm


def hydrodynamic_forces(lat, f, X, Av, nrm, probe=1.2):
    """Eqs. hydroForP / hydroForNu: F_p = -(p+ - p-) n A and
    F_tau = (tau+ - tau-) . n A, with p = c_s^2 rho and
    tau = rho nu (grad u + grad u^T) taken at X +- 1.2 dx n by MLS (Reading S-d)."""
    nu = viscosity(lat.tau)
    out = []
    for sgn in (+1.0, -1.0):
        P = X + sgn * probe * nrm
        st = ib.stencil(lat, P)
        flat = st.nodes.reshape(-1)
        rho_k = ib.node_density(f, flat).reshape(st.nodes.shape)
        u_k = ib.node_velocity(f, flat).reshape(st.nodes.shape + (3,))
        rho = np.einsum("mk,mk->m", st.phi, rho_k)
        G = np.einsum("mjk,mkc->mcj", st.grad, u_k)   # G[m, c, j] = d u_c / d x_j
        tau = rho[:, None, None] * nu * (G + np.transpose(G, (0, 2, 1)))
        out.append((rho / 3.0, tau))
    (pp, tp), (pm, tm) = out
    Fp = -((pp - pm) * Av)[:, None] * nrm
    Ft = np.einsum("mij,mj->mi", tp - tm, nrm) * Av[:, None]
    return Fp, Ft


def repulsion_forces(Xs, nrms, u_max, cutoff=2.0):
    """Eq. collision between markers of different bodies closer than the
    cutoff (Reading S-e): F_i = u_max dt/(8 sqrt 2) sqrt(dx / d^5) n^-_i, summed
    over the partners j, n^- the inward normal of marker i."""
    c = u_max / (8.0 * math.sqrt(2.0))
    out = [np.zeros(X.shape, dtype=np.result_type(X, c, nrms[k])) for k, X in enumerate(Xs)]
    lo = [np.real(X).min(axis=0) for X in Xs]
    hi = [np.real(X).max(axis=0) for X in Xs]
    for a in range(len(Xs)):
        for b in range(len(Xs)):
            if a == b:
                continue
            # bodies whose bounding boxes are farther apart than the cutoff
            # have no marker pair within it
            if np.any(lo[a] - hi[b] >= cutoff) or np.any(lo[b] - hi[a] >= cutoff):
                continue
            d = _norm(Xs[a][:, None, :] - Xs[b][None, :, :], axis=2)
            near = np.real(d) < cutoff
            w = np.zeros(d.shape, dtype=np.result_type(d, c))
            w[near] = c * np.sqrt(1.0 / d[near] ** 5)
            out[a] += -w.sum(axis=1)[:, None] * nrms[a]
    return out


def diagnostics(X, tris):
    """FP64 capsule reductions: enclosed volume (divergence theorem, tetrahedra
    fanned from the vertex mean), surface area, volume centroid, the volume
    second-moment tensor about the centroid and the Taylor deformation index
    D = (a_max - a_min)/(a_max + a_min) of the equivalent ellipsoid
    (a_i = sqrt(5 lambda_i / V)); Reading R."""
    X = np.asarray(X)
    tris = np.asarray(tris, dtype=np.int64)
    o = X.mean(axis=0)
    a, b, c = X[tris[:, 0]] - o, X[tris[:, 1]] - o, X[tris[:, 2]] - o
    v = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    V = v.sum()
    S = 0.5 * _norm(np.cross(b - a, c - a), axis=1).sum()
    s = a + b + c
    cen_rel = (v[:, None] * s / 4.0).sum(axis=0) / V
    M2 = np.einsum("t,tij->ij", v / 20.0,
                   np.einsum("ti,tj->tij", a, a) + np.einsum("ti,tj->tij", b, b)
                   + np.einsum("ti,tj->tij", c, c) + np.einsum("ti,tj->tij", s, s))
    C = M2 - V * np.outer(cen_rel, cen_rel)
    lam = _eigvalsh(C)
    q = 5.0 * lam / V
    ax = np.sqrt(np.where(np.real(q) > 0.0, q, 0.0))
    hi, lo = ax[np.argmax(np.real(ax))], ax[np.argmin(np.real(ax))]
    D = (hi - lo) / (hi + lo)
    return dict(volume=V, area=S, centroid=o + cen_rel, second_moment=C, semi_axes=ax, taylor_D=D)


def max_stretch(X, rest):
    e = rest.topo.edge
    l = _norm(X[e[:, 0]] - X[e[:, 1]], axis=1)
    return float(np.max(np.real(l / rest.l0)))
