"""Discrete adjoint (reverse mode) of the oracle's lattice step, FP64.

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.

The forward map of one step is the oracle's own ``Lattice.step`` (Eq. evoleq
collide + stream, Eq. bbouzidi wall links, Eq. extbound faces) on a lattice
without capsules.  Its adjoint is assembled here without any derivative worked
out by hand:

* every local Jacobian (the collision at a node, the wall rule of a link, the
  face rule at a face node, the objective at a node) is probed from the forward
  oracle functions by the complex step, d g(x)/dx . v = Im g(x + i h v) / h,
  which is exact to rounding for these rational maps;
* the data movement is transposed explicitly: the pull stream becomes a push,
  the wall rule's reads become scatter-adds.

Objective: J = sum over the fluid nodes of a box of d . u at the final step,
u = (sum f e + F/2) / rho (bullets below Eq. evoleq).  Parameters:
  s_u : the inlet velocities scale as u_w (1 + s_u)   (dJ/du_max = dJ/ds_u / u_max)
  s_q : the wall-link distances move as q + s_q dq    (dq = dq/dr_j of the links:
        dJ/dr_j = dJ/ds_q; the fluid/solid tags are held fixed)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lattice import Lattice, OPP, bouzidi_value, collide, moments

H = 1e-30      # complex-step size


@dataclass
class Objective:
    lo: tuple          # box lower corner (x, y, z), inclusive
    hi: tuple          # box upper corner, exclusive
    d: tuple           # weights of (u_x, u_y, u_z)

    def nodes(self, lat: Lattice):
        sel = lat.fluid.copy()
        for c, a, b in ((lat.X, self.lo[0], self.hi[0]), (lat.Y, self.lo[1], self.hi[1]),
                        (lat.Z, self.lo[2], self.hi[2])):
            sel &= (c >= a) & (c < b)
        return np.nonzero(sel)[0]


def objective(lat: Lattice, f, obj: Objective) -> float:
    n = obj.nodes(lat)
    F = lat.force_field(None)[n]
    _, u = moments(f[:, n], F)
    return float((u @ np.asarray(obj.d, dtype=np.float64)).sum())


def objective_grad(lat: Lattice, f, obj: Objective):
    """dJ/df (19, N), probed direction by direction."""
    n = obj.nodes(lat)
    F = lat.force_field(None)[n]
    d = np.asarray(obj.d, dtype=np.float64)
    g = np.zeros((19, lat.N))
    for j in range(19):
        fc = f[:, n].astype(np.complex128)
        fc[j] += 1j * H
        _, u = moments(fc, F)
        g[j, n] = (u @ d).imag / H
    return g


def collide_vjp(lat: Lattice, f, lam_star):
    """Adjoint of the collision at every fluid node: (df*/df)^T lam*."""
    fl = lat.fluid
    F = lat.force_field(None)[fl]
    out = np.zeros_like(lam_star)
    base = f[:, fl].astype(np.complex128)
    for j in range(19):
        fc = base.copy()
        fc[j] += 1j * H
        col = collide(fc, F, lat.tau).imag / H        # d f*_k / d f_j, (19, n_fluid)
        out[j, fl] = (col * lam_star[:, fl]).sum(axis=0)
    return out


def stream_vjp(lat: Lattice, lam_s):
    """Adjoint of the pull stream: the value pulled into (i, n) from
    (i, n - e_i) is pushed back."""
    out = np.zeros_like(lam_s)
    for i in range(19):
        ok = lat.fluid & lat.src_ok[i] & lat.fluid[lat.src[i]]
        np.add.at(out[i], lat.src[i][ok], lam_s[i, ok])
    return out


def bfl_vjp(lat: Lattice, lam_b, fstar, dq):
    """Adjoint of the wall links: the value written to (ib, x_b) is a linear
    combination of five post-collision values; returns their adjoint and
    dJ/ds_q = sum over links of lam(ib, x_b) d(value)/dq dq."""
    out = np.zeros_like(lam_b)
    if lat.links_node.size == 0:
        return out, 0.0
    xb, i, ib, m1, ok1, m2, ok2 = lat.link_neighbours()
    q = lat.links_q
    z1 = np.where(ok1, m1, 0)
    z2 = np.where(ok2, m2, 0)
    args = [fstar[i, xb], np.where(ok1, fstar[i, z1], 0.0), np.where(ok2, fstar[i, z2], 0.0),
            fstar[ib, xb], np.where(ok1, fstar[ib, z1], 0.0)]
    lam = lam_b[ib, xb]
    targets = [(i, xb, None), (i, z1, ok1), (i, z2, ok2), (ib, xb, None), (ib, z1, ok1)]
    for a, (rows, cols, mask) in enumerate(targets):
        probe = [v.astype(np.complex128) for v in args]
        probe[a] = probe[a] + 1j * H
        c = bouzidi_value(q, *probe, ok1, ok2).imag / H
        w = c * lam if mask is None else np.where(mask, c * lam, 0.0)
        np.add.at(out, (rows, cols), w)
    dval = bouzidi_value(q + 1j * H * np.asarray(dq, dtype=np.float64), *args, ok1, ok2).imag / H
    return out, float((lam * dval).sum())


def zh_vjp(lat: Lattice, lam_z, fnew_b):
    """Adjoint of the face rule at every face node (identity elsewhere) and
    dJ/ds_u through the imposed inlet velocities."""
    out = lam_z.copy()
    nodes = []
    for face, spec in enumerate(lat.faces):
        if spec is None or spec.kind == 0:
            continue
        nd, _ = lat.face_nodes(face)
        nodes.append(nd)
    if not nodes:
        return out, 0.0
    nodes = np.concatenate(nodes)
    base = np.nan_to_num(fnew_b).astype(np.complex128)
    for j in range(19):
        fc = base.copy()
        fc[j, nodes] += 1j * H
        lat.zou_he(fc)
        col = fc.imag[:, nodes] / H                     # d out_k / d in_j at the face nodes
        out[j, nodes] = (col * lam_z[:, nodes]).sum(axis=0)
    # inlet velocities scaled by (1 + s_u)
    saved = lat.faces
    try:
        lat.faces = [spec if (spec is None or spec.kind != 1) else
                     type(spec)(spec.kind, spec.rho, np.asarray(spec.velocity, dtype=np.float64) * (1.0 + 1j * H))
                     for spec in saved]
        fc = base.copy()
        lat.zou_he(fc)
        dsu = float((fc.imag[:, nodes] / H * lam_z[:, nodes]).sum())
    finally:
        lat.faces = saved
    return out, dsu


def gradient(lat: Lattice, f0, steps, obj: Objective, dq):
    """J(f^steps) and (dJ/ds_u, dJ/ds_q) by the discrete adjoint of `steps`
    oracle steps from f0 (no capsules, no IB force)."""
    fs = [np.array(f0, dtype=np.float64)]
    for _ in range(steps):
        fs.append(lat.step(fs[-1]))
    J = objective(lat, fs[-1], obj)
    lam = objective_grad(lat, fs[-1], obj)
    g_u = 0.0
    g_q = 0.0
    solid = ~lat.fluid
    for t in reversed(range(steps)):
        f = fs[t]
        fstar = lat.collide_all(f, None)
        fb = lat.bouzidi(lat.stream(fstar), fstar)
        lam[:, solid] = 0.0                             # solid columns are reset to w
        lam_b, du = zh_vjp(lat, lam, fb)
        g_u += du
        lam_star, dqs = bfl_vjp(lat, lam_b, fstar, dq)
        g_q += dqs
        lam_star += stream_vjp(lat, lam_b)
        lam = collide_vjp(lat, f, lam_star)
    return J, g_u, g_q


def perturbed(lat: Lattice, s_u=0.0, s_q=0.0, dq=None) -> Lattice:
    """A copy of the lattice with inlet velocities u_w (1 + s_u) and link
    distances q + s_q dq (for finite-difference checks)."""
    import copy
    out = copy.copy(lat)
    out.faces = [spec if (spec is None or spec.kind != 1) else
                 type(spec)(spec.kind, spec.rho, np.asarray(spec.velocity, dtype=np.float64) * (1.0 + s_u))
                 for spec in lat.faces]
    if dq is not None and s_q != 0.0:
        out.links_q = lat.links_q + s_q * np.asarray(dq, dtype=np.float64)
    return out


def value(lat: Lattice, f0, steps, obj: Objective) -> float:
    f = np.array(f0, dtype=np.float64)
    for _ in range(steps):
        f = lat.step(f)
    return objective(lat, f, obj)


# ---------------------------------------------------------------------------
# The coupled step with capsules: derivative of a capsule objective
# ---------------------------------------------------------------------------
# Objective of the capsule adjoint: J = w_D D + w_off (y_c - y_sym) of capsule 0
# after the last step, with D the Taylor deformation index and y_c the y
# coordinate of the volume centroid (the branch offset from the symmetry plane
# y_sym), both from membrane.diagnostics.  Parameters: the capillary number Ca
# of capsule 0 (k_s0 = rho nu u_ref / Ca, u_ref held fixed), the peak inlet
# velocity u_max (the inlet data scale as u_w (1 + s), dJ/du_max = dJ/ds /
# u_max; u_ref and the repulsion coefficient are held fixed), and the
# junction radius r_j (the link distances move as q + s dq with dq = dq/dr_j,
# tags fixed).  The derivative of the whole discrete run comes from the
# complex step: the forward oracle is run once per parameter with that
# parameter perturbed by i h, every discrete decision taken on real parts,
# and dJ/dp = Im J / h, exact to rounding for this smooth map.

def capsule_objective(body, w_D, w_off, y_sym=0.0):
    from . import membrane
    d = membrane.diagnostics(body.x, body.tris)
    return w_D * d["taylor_D"] + w_off * (d["centroid"][1] - y_sym)


def coupled_run(case, steps, w_D=1.0, w_off=0.0, y_sym=0.0, dCa=0.0, ds_u=0.0, ds_q=0.0):
    """J after `steps` coupled oracle steps of a case (geometry, tau, u_max,
    capsules, with wall links carrying dq), with Ca of capsule 0 moved by dCa,
    the inlet data scaled by (1 + ds_u) and the link distances moved by
    ds_q * dq.  Any of the moves may be complex."""
    from .lattice import Lattice
    from .sim import Simulation
    g = case["geometry"]
    lat = Lattice(g.nx, g.ny, g.nz, case["tau"], g.tag, g.links, g.faces, g.periodic,
                  body_force=case.get("body_force", (0.0, 0.0, 0.0)))
    lat = perturbed(lat, s_u=ds_u, s_q=ds_q, dq=g.links["dq"])
    cplx = any(np.iscomplexobj(np.asarray(v)) for v in (dCa, ds_u, ds_q))
    o = Simulation(lat, u_max=case["u_max"])
    if cplx:
        o.f = o.f.astype(np.complex128)
    for k, c in enumerate(case["capsules"]):
        params = dict(c["params"])
        if k == 0:
            params["Ca"] = params["Ca"] + dCa
        o.add_body(c["verts"], c["tris"], params, c.get("vel0"))
    o.step(steps)
    return capsule_objective(o.bodies[0], w_D, w_off, y_sym), o


def coupled_gradient(case, steps, w_D=1.0, w_off=0.0, y_sym=0.0, h=1e-30):
    """J and (dJ/dCa, dJ/du_max, dJ/dr_j) of `steps` coupled oracle steps by
    the complex step (one complex run per parameter)."""
    J, _ = coupled_run(case, steps, w_D, w_off, y_sym)
    g_ca = np.imag(coupled_run(case, steps, w_D, w_off, y_sym, dCa=1j * h)[0]) / h
    g_su = np.imag(coupled_run(case, steps, w_D, w_off, y_sym, ds_u=1j * h)[0]) / h
    g_sq = np.imag(coupled_run(case, steps, w_D, w_off, y_sym, ds_q=1j * h)[0]) / h
    return float(np.real(J)), float(g_ca), float(g_su / case["u_max"]), float(g_sq)
