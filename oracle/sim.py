"""FP64 oracle of the whole coupled time step, in the order
  1. immersed-boundary pre-pass on the fluid solution at t: MLS interpolation
     of u* at the markers, F_l = (U_b - U_l)/dt, spreading to f_ib
                                                            (Eqs. uLag .. bodyforce)
  2. structure forces F^tot(t) at x(t) from the same field  (Eqs. strainFor .. collision)
  3. Verlet (soft) or Newton-Euler (rigid) update, with the tentative
     velocity u_v,0 = U_l of step 1                         (Eqs. verletPos .. angularVelRig)
  4. collide, stream, BFL wall links, Zou-He faces          (Eqs. evoleq, extbound, bbouzidi)
  5. damage check: an edge at twice its rest length stops the run
(Reading T1 for the order, which the paper does not state: every structure
quantity of the step is taken from the fluid solution at time t, the field the
IB pre-pass interpolates.  Interpolating u_v,0 and the probes from the field
after the collision instead makes the explicit coupled scheme grow a
period-2 tangential membrane mode at Re = 10-20.)

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.
"""
from __future__ import annotations

import math

import numpy as np

from . import ib, membrane
from .lattice import Lattice


def rotation_matrix(w):
    """Rotation by the vector angle w (Rodrigues)."""
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.eye(3)
    k = w / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1.0 - math.cos(th)) * (K @ K)


def verlet(x, x_prev, uv0, F, mv):
    """Eqs. verletPos, verletVel, verletPosC with dt = 1:
    predictor x* = x + u_v,0 + F/(2 m_v); u = (3/2 x* - 2 x + 1/2 x_prev);
    corrector x(t+dt) = x + u + F/(2 m_v).  Returns (x(t+dt), u(t+dt))."""
    acc = 0.5 * F / mv
    x_pred = x + uv0 + acc
    u_new = 1.5 * x_pred - 2.0 * x + 0.5 * x_prev
    return x + u_new + acc, u_new


def rigid_velocity(v1, v2, vdot):
    """Eq. angularVelRig with dt = 1: v(t) = 2/3 (2 v(t-dt) - 1/2 v(t-2dt) + vdot)."""
    return (2.0 / 3.0) * (2.0 * v1 - 0.5 * v2 + vdot)


class Body:
    """One capsule: rest data plus state x(t), x(t-dt), vertex velocity, and
    the rigid centre/velocities (Reading S-f for the start values)."""

    def __init__(self, X0, tris, params, tau, vel0=None):
        self.rest = membrane.CapsuleRest(X0, tris, params, tau)
        self.tris = np.asarray(tris, dtype=np.int64)
        self.x = np.array(X0, dtype=np.float64)
        self.x_prev = self.x.copy()
        v0 = np.zeros(3) if vel0 is None else np.asarray(vel0, dtype=np.float64)
        self.vel = np.tile(v0, (self.x.shape[0], 1))
        self.rigid = self.rest.rigid
        self.xc = membrane.diagnostics(self.x, self.tris)["centroid"]
        self.u1 = v0.copy()     # u(t - dt)
        self.u2 = v0.copy()     # u(t - 2 dt)
        self.w1 = np.zeros(3)
        self.w2 = np.zeros(3)
        self.inertia = 0.4 * self.rest.mass * self.rest.radius ** 2   # Reading S-g

    def boundary_velocity(self):
        """U_b of the markers: the vertex velocity (soft) or u + w x r (rigid)."""
        if self.rigid:
            return self.u1[None, :] + np.cross(self.w1[None, :], self.x - self.xc[None, :])
        return self.vel


class Simulation:
    def __init__(self, lat: Lattice, f0=None, u_max=0.02):
        self.lat = lat
        self.f = lat.init_equilibrium() if f0 is None else np.array(f0, dtype=np.float64)
        self.bodies = []
        self.u_max = float(u_max)
        self.t = 0
        self.damaged = False
        self.last = {}

    def add_body(self, X0, tris, params, vel0=None):
        self.bodies.append(Body(X0, tris, params, self.lat.tau, vel0))
        return len(self.bodies) - 1

    def ib_force(self):
        """Step 1: f_ib on the lattice and per-body marker data."""
        lat = self.lat
        f_ib = np.zeros((lat.N, 3))
        per = []
        for b in self.bodies:
            st = ib.stencil(lat, b.x)
            U = ib.interpolate_velocity(self.f, st)
            Fl = b.boundary_velocity() - U          # (U_b - U)/dt
            Av, nrm = membrane.vertex_areas_normals(b.x, b.tris, b.x.shape[0])
            f_ib = f_ib + ib.spread(lat.N, st, Fl, Av)
            per.append(dict(stencil=st, U=U, F=Fl, Av=Av, nrm=nrm))
        return f_ib, per

    def structure(self, fnew, per):
        """Step 2: total force F^tot(t) on each vertex at x(t); the probes read
        the populations passed in (the solution at t)."""
        lat = self.lat
        Fs = []
        nrms = [p["nrm"] for p in per]
        rep = membrane.repulsion_forces([b.x for b in self.bodies], nrms, self.u_max) \
            if len(self.bodies) > 1 else [np.zeros_like(b.x) for b in self.bodies]
        for b, p, Fr in zip(self.bodies, per, rep):
            Av, nrm = p["Av"], p["nrm"]
            Fp, Ft = membrane.hydrodynamic_forces(lat, fnew, b.x, Av, nrm)
            F = Fp + Ft + Fr
            if not b.rigid:
                V = membrane.diagnostics(b.x, b.tris)["volume"]
                F = F + membrane.stretch_forces(b.x, b.rest) + membrane.bending_forces(b.x, b.rest) \
                    + membrane.volume_forces(b.x, b.rest, V, Av, nrm)
            Fs.append(F)
            p["F_tot"] = F
        return Fs

    def update(self, fnew, per, Fs):
        """Step 3: Eqs. verletPos, verletVel, verletPosC (soft) or the
        Newton-Euler system with Eq. angularVelRig (rigid)."""
        for b, p, F in zip(self.bodies, per, Fs):
            if b.rigid:
                r = b.x - b.xc[None, :]
                Ftot = F.sum(axis=0)
                Mtot = np.cross(r, F).sum(axis=0)
                udot = Ftot / b.rest.mass
                wdot = Mtot / b.inertia
                u = rigid_velocity(b.u1, b.u2, udot)
                w = rigid_velocity(b.w1, b.w2, wdot)
                R = rotation_matrix(w)
                xc_new = b.xc + u
                b.x_prev = b.x.copy()
                b.x = xc_new[None, :] + r @ R.T
                b.xc = xc_new
                b.u2, b.u1 = b.u1, u
                b.w2, b.w1 = b.w1, w
                b.vel = b.boundary_velocity()
            else:
                # u_v,0(t + dt): the fluid velocity interpolated at x(t) by the
                # IB pre-pass (Eq. uLag on the solution at t)
                uv0 = p["U"]
                p["uv0"] = uv0
                x_new, u_new = verlet(b.x, b.x_prev, uv0, F, b.rest.mv)
                b.x_prev = b.x
                b.x = x_new
                b.vel = u_new

    def step(self, n=1):
        done = 0
        for _ in range(n):
            if self.damaged:
                break
            f_ib, per = self.ib_force()
            Fs = self.structure(self.f, per)
            self.update(self.f, per, Fs)
            self.f = self.lat.step(self.f, f_ib if self.bodies else None)
            self.t += 1
            done += 1
            self.last = dict(f_ib=f_ib, per=per)
            for b in self.bodies:
                if not b.rigid and membrane.max_stretch(b.x, b.rest) >= 2.0:
                    self.damaged = True
        return done

    def stats(self, k):
        b = self.bodies[k]
        d = membrane.diagnostics(b.x, b.tris)
        d["dS"] = (d["area"] - b.rest.S0) / b.rest.S0
        d["max_stretch"] = membrane.max_stretch(b.x, b.rest)
        return d
