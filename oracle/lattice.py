"""FP64 lattice part of the oracle: D3Q19 BGK with Guo forcing, pull
streaming, quadratic Bouzidi-Firdaouss-Lallemand bounce-back, Zou-He faces.

TEST INFRASTRUCTURE (see the package docstring): never imported by the product.

Distribution array layout: f[i, node], i in the numbering of Eq. e_i,
node = x + nx*(y + ny*z).
"""
from __future__ import annotations

import numpy as np

# Eq. e_i (Section "Fluid evolution"): the 19 lattice velocities, e_0 ... e_18.
E = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0],
    [0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1],
    [0, 0, 0, 0, 0, 1, -1, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, 1, -1],
], dtype=np.int64).T
Ef = E.astype(np.float64)
# Weights below Eq. eqfunc: omega_0 = 1/3, omega_1-6 = 1/18, omega_7-18 = 1/36.
W = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
# c_s = 1/sqrt(3)  (below Eq. evoleq)
CS2 = 1.0 / 3.0
# opposite direction: e_opp(i) = -e_i
OPP = np.array([int(np.nonzero((E == -E[i]).all(axis=1))[0][0]) for i in range(19)])

FACE_NORMALS = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]])
FACE_VELOCITY = 1
FACE_PRESSURE = 2


def viscosity(tau):
    """nu = c_s^2 (tau - dt/2)  (below Eq. evoleq)."""
    return CS2 * (tau - 0.5)


def equilibrium(rho, u):
    """Eq. eqfunc: f_i^eq = w_i rho [1 + e.u/c_s^2 + (e.u)^2/(2 c_s^4) - u^2/(2 c_s^2)].
    rho (N,), u (N,3) -> (19, N)."""
    eu = Ef @ u.T
    usq = np.einsum("nj,nj->n", u, u)
    return W[:, None] * rho[None, :] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2)
                                        - usq[None, :] / (2.0 * CS2))


def guo_forcing(u, F, tau):
    """Eq. forcing: F_i = (1 - 1/(2 tau)) w_i [(e_i - u)/c_s^2 + (e_i.u) e_i/c_s^4] . F.
    u, F (N,3) -> (19, N)."""
    eu = Ef @ u.T
    eF = Ef @ F.T
    uF = np.einsum("nj,nj->n", u, F)
    return (1.0 - 0.5 / tau) * W[:, None] * ((eF - uF[None, :]) / CS2 + eu * eF / (CS2 * CS2))


def moments(f, F):
    """rho = sum_i f_i ; rho u = sum_i f_i e_i + (dt/2) f_ib  (bullets below Eq. evoleq).
    f (19, N), F (N,3) -> rho (N,), u (N,3)."""
    rho = f.sum(axis=0)
    mom = (Ef.T @ f).T
    u = (mom + 0.5 * F) / rho[:, None]
    return rho, u


def collide(f, F, tau):
    """Right-hand side of Eq. evoleq: f* = f - (dt/tau)(f - f^eq) + dt F_i, with
    the force-corrected u in both f^eq and F_i (Reading T2)."""
    rho, u = moments(f, F)
    feq = equilibrium(rho, u)
    return f - (f - feq) / tau + guo_forcing(u, F, tau)


def bouzidi_value(q, fi_b, fi_1, fi_2, fib_b, fib_1, ok1, ok2):
    """The returning population f_ib(x_b, t+1) of one wall link (Eq. bbouzidi
    with the q >= 1/2 branch of Reading B and the fall-backs of Reading B'),
    from the post-collision values f*_i at x_b, x_b - e_i, x_b - 2e_i and
    f*_ib at x_b, x_b - e_i; ok1 / ok2 say whether x_b - e_i / x_b - 2e_i are
    fluid."""
    small = np.real(q) < 0.5          # the branch is taken on the real link distance
    quad_s = q * (2 * q + 1) * fi_b + (1 - 4 * q * q) * fi_1 - q * (1 - 2 * q) * fi_2
    lin_s = 2 * q * fi_b + (1 - 2 * q) * fi_1
    val_s = np.where(ok1 & ok2, quad_s, np.where(ok1, lin_s, fi_b))
    quad_l = fi_b / (q * (2 * q + 1)) + (2 * q - 1) / q * fib_b + (1 - 2 * q) / (1 + 2 * q) * fib_1
    lin_l = fi_b / (2 * q) + (2 * q - 1) / (2 * q) * fib_b
    val_l = np.where(ok1, quad_l, lin_l)
    return np.where(small, val_s, val_l)


class Lattice:
    """Box lattice with fluid/solid tags, wall links and face conditions.

    Parameters mirror the C-ABI: tag (N,) uint8 (0 fluid / 1 solid); links with
    fields node, dir, q (dir = direction from the fluid node toward the wall);
    faces = list of 6 objects with .kind / .rho / .velocity (face layout of the
    geometry module); periodic (3 bools); body_force (3,) added to f_ib."""

    def __init__(self, nx, ny, nz, tau, tag, links, faces, periodic, body_force=(0.0, 0.0, 0.0)):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.tau = float(tau)
        self.tag = np.asarray(tag, dtype=np.uint8).reshape(-1)
        self.fluid = self.tag == 0
        self.periodic = tuple(bool(p) for p in periodic)
        self.body_force = np.asarray(body_force, dtype=np.float64)
        self.links_node = np.asarray(links["node"], dtype=np.int64)
        self.links_dir = np.asarray(links["dir"], dtype=np.int64)
        self.links_q = np.asarray(links["q"], dtype=np.float64)
        self.faces = faces
        n = np.arange(self.N, dtype=np.int64)
        self.X = n % self.nx
        self.Y = (n // self.nx) % self.ny
        self.Z = n // (self.nx * self.ny)
        # pull sources: node - e_i, with wrap on periodic axes
        self.src = np.zeros((19, self.N), dtype=np.int64)
        self.src_ok = np.zeros((19, self.N), dtype=bool)
        for i in range(19):
            idx, ok = self.shift(n, -E[i])
            self.src[i] = idx
            self.src_ok[i] = ok

    # -- indexing helpers ---------------------------------------------------
    def shift(self, nodes, d):
        """Index of nodes + d (d integer 3-vector), and whether it lies in the
        domain (periodic axes wrap)."""
        nodes = np.asarray(nodes, dtype=np.int64)
        X = nodes % self.nx
        Y = (nodes // self.nx) % self.ny
        Z = nodes // (self.nx * self.ny)
        out = []
        ok = np.ones(nodes.shape, dtype=bool)
        for c, dc, n, per in ((X, d[0], self.nx, self.periodic[0]),
                              (Y, d[1], self.ny, self.periodic[1]),
                              (Z, d[2], self.nz, self.periodic[2])):
            s = c + int(dc)
            if per:
                s = s % n
            else:
                ok &= (s >= 0) & (s < n)
                s = np.clip(s, 0, n - 1)
            out.append(s)
        return out[0] + self.nx * (out[1] + self.ny * out[2]), ok

    def is_fluid(self, nodes, ok):
        return ok & self.fluid[np.where(ok, nodes, 0)]

    def face_nodes(self, face):
        """Fluid nodes on a face and their index in the face layout."""
        ax = face // 2
        coord = (self.X, self.Y, self.Z)[ax]
        lim = 0 if face % 2 == 0 else (self.nx, self.ny, self.nz)[ax] - 1
        nodes = np.nonzero(self.fluid & (coord == lim))[0]
        if ax == 0:
            fidx = self.Y[nodes] + self.ny * self.Z[nodes]
        elif ax == 1:
            fidx = self.X[nodes] + self.nx * self.Z[nodes]
        else:
            fidx = self.X[nodes] + self.nx * self.Y[nodes]
        return nodes, fidx

    # -- the step -----------------------------------------------------------
    def force_field(self, f_ib):
        F = np.zeros((self.N, 3)) if f_ib is None else np.array(f_ib)
        return F + self.body_force[None, :]

    def collide_all(self, f, f_ib):
        F = self.force_field(f_ib)
        fstar = np.array(f, dtype=np.result_type(f, F, np.float64), copy=True)
        fl = self.fluid
        fstar[:, fl] = collide(f[:, fl], F[fl], self.tau)
        return fstar

    def stream(self, fstar):
        """f_i(x + e_i, t+dt) = f*_i(x, t) (Eq. evoleq, streaming phase), as a
        pull from fluid sources; populations with no fluid source are left NaN
        for the wall and face conditions to fill."""
        fnew = np.full_like(fstar, np.nan)
        for i in range(19):
            ok = self.fluid & self.src_ok[i] & self.fluid[self.src[i]]
            fnew[i, ok] = fstar[i, self.src[i][ok]]
        return fnew

    def bouzidi(self, fnew, fstar):
        """Eq. bbouzidi with the q >= 1/2 branch re-derived by quadratic
        interpolation (Reading B): for a link (x_b, i, q) with x_b + e_i solid,
            q <  1/2: f_ib(x_b) = q(2q+1) f*_i(x_b) + (1-4q^2) f*_i(x_b-e_i) - q(1-2q) f*_i(x_b-2e_i)
            q >= 1/2: f_ib(x_b) = f*_i(x_b)/(q(2q+1)) + (2q-1)/q f*_ib(x_b) + (1-2q)/(1+2q) f*_ib(x_b-e_i)
        (ib = opposite of i).  Missing upstream fluid nodes fall back to the
        two-point rule, then to halfway bounce-back (Reading B')."""
        if self.links_node.size == 0:
            return fnew
        xb, i, ib, m1, ok1, m2, ok2 = self.link_neighbours()
        q = self.links_q
        fi_b = fstar[i, xb]
        fib_b = fstar[ib, xb]
        fi_1 = np.where(ok1, fstar[i, np.where(ok1, m1, 0)], 0.0)
        fi_2 = np.where(ok2, fstar[i, np.where(ok2, m2, 0)], 0.0)
        fib_1 = np.where(ok1, fstar[ib, np.where(ok1, m1, 0)], 0.0)
        fnew[ib, xb] = bouzidi_value(q, fi_b, fi_1, fi_2, fib_b, fib_1, ok1, ok2)
        return fnew

    def link_neighbours(self):
        """Per wall link (x_b, i): x_b, i, the opposite direction ib, the nodes
        x_b - e_i and x_b - 2 e_i and whether they are fluid."""
        xb = self.links_node
        i = self.links_dir
        ib = OPP[i]
        m1 = np.empty_like(xb)
        ok1 = np.empty(xb.shape, dtype=bool)
        m2 = np.empty_like(xb)
        ok2 = np.empty(xb.shape, dtype=bool)
        for d in range(1, 19):
            sel = i == d
            if not sel.any():
                continue
            a, oka = self.shift(xb[sel], -E[d])
            b, okb = self.shift(xb[sel], -2 * E[d])
            m1[sel], ok1[sel] = a, self.is_fluid(a, oka)
            m2[sel], ok2[sel] = b, self.is_fluid(b, okb)
        return xb, i, ib, m1, ok1, m2, ok2

    def zou_he(self, fnew):
        """Eq. extbound generalised to the six faces through the velocity
        vectors (Readings Z, Z', Z''): with n the outward normal of the face,
            rho = [sum_{e.n=0} f + 2 sum_{e.n>0} f] / (1 + u.n)
        (velocity face), or u = u_n n with u_n from the same balance (pressure
        face); then every population entering from outside (e.n < 0) is
            e = -n     : f = f_opp - rho u.n / 3
            e = -n + t : f = f_opp - rho u.n / 6 + rho u.t / 6 - N_t,
                         N_t = (1/2) sum_{e.n=0} f (e.t) - rho u.t / 3."""
        for face, spec in enumerate(self.faces):
            if spec is None or spec.kind == 0:
                continue
            nodes, fidx = self.face_nodes(face)
            if nodes.size == 0:
                continue
            nrm = FACE_NORMALS[face]
            en = E @ nrm
            K0 = np.nonzero(en == 0)[0]
            Kp = np.nonzero(en > 0)[0]
            Km = np.nonzero(en < 0)[0]
            S = fnew[K0][:, nodes].sum(axis=0) + 2.0 * fnew[Kp][:, nodes].sum(axis=0)
            if spec.kind == FACE_VELOCITY:
                uw = np.asarray(spec.velocity)[fidx].astype(np.result_type(spec.velocity, np.float64))
                un = uw @ nrm
                rho = S / (1.0 + un)
            else:
                rho = np.full(nodes.shape, float(spec.rho))
                un = S / rho - 1.0
                uw = un[:, None] * nrm[None, :].astype(np.float64)
            for k in Km:
                t = E[k] + nrm
                fo = fnew[OPP[k], nodes]
                if not t.any():
                    fnew[k, nodes] = fo - rho * un / 3.0
                else:
                    ut = uw @ t
                    Nt = 0.5 * (fnew[K0][:, nodes] * (E[K0] @ t)[:, None]).sum(axis=0) - rho * ut / 3.0
                    fnew[k, nodes] = fo - rho * un / 6.0 + rho * ut / 6.0 - Nt
        return fnew

    def step(self, f, f_ib=None, check=True):
        """One step in the oracle order: collide, stream, wall links, faces."""
        fstar = self.collide_all(f, f_ib)
        fnew = self.stream(fstar)
        self.bouzidi(fnew, fstar)
        self.zou_he(fnew)
        if check:
            miss = np.isnan(fnew[:, self.fluid])
            if miss.any():
                raise RuntimeError(f"{int(miss.sum())} populations left unset after the boundary conditions")
        fnew[:, ~self.fluid] = W[:, None]
        return fnew

    # -- initial state and read-out ----------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        rho = np.ones(self.N) if rho is None else np.asarray(rho, dtype=np.float64)
        u = np.zeros((self.N, 3)) if u is None else np.asarray(u, dtype=np.float64)
        return equilibrium(rho, u)

    def macroscopic(self, f, include_body_force=True):
        """rho and u of the bullets below Eq. evoleq, with the uniform body force
        (the only force present between steps) in the momentum."""
        F = np.zeros((self.N, 3))
        if include_body_force:
            F += self.body_force[None, :]
        rho, u = moments(f, F)
        rho = np.where(self.fluid, rho, 0.0)
        u = np.where(self.fluid[:, None], u, 0.0)
        return rho, u
