"""Pins of oracle parts that the other CPU tests leave open: the rigid-body
Newton-Euler update, the viscous probe stress, the mass balance of the Zou-He
faces in a steady duct, the duct flow at D = 24, and the momentum exchange of
a free rigid sphere with the fluid.  Each expected value is
worked out here by hand from the closed form, not by calling the oracle's own
formula (no GPU)."""
import math

import numpy as np
import pytest

from oracle import lattice as L
from oracle import membrane, sim
from paper_2207_06043_gb300 import geometry as G


# ---------------------------------------------------------------------------
# Rigid body (Section "Rigid structures transport", Eq. angularVelRig)
# ---------------------------------------------------------------------------
def octahedron():
    """Unit octahedron, outward counter-clockwise triangles."""
    X = np.array([(1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)], dtype=np.float64)
    T = np.array([(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4), (1, 0, 5), (2, 1, 5), (3, 2, 5), (0, 3, 5)])
    return X, T


def test_rigid_newton_euler_three_steps_by_hand():
    """A rigid octahedron under a uniform force f (along y, no torque) and a
    couple of two tangential forces k z x r at vertices 0 and 2 (torque 2 k z,
    no net force), both re-applied at the current positions every step.

    By hand, with dt = 1 and u(-dt) = u(-2dt) = 0, Eq. angularVelRig gives
    u_1 = 2/3 a, u_2 = 2/3 (2 u_1 + a) = 14/9 a, u_3 = 2/3 (2 u_2 - u_1/2 + a)
    = 68/27 a for a constant acceleration a, and the same for omega with the
    angular acceleration.  Mass = 1.1 V0 with V0 = 4/3, inertia 0.4 m r^2 with
    r the radius of the sphere of volume V0 (Reading S-g).  Vertex 0 starts at
    +x and turns counter-clockwise about +z: (cos th, sin th, 0) about the
    centre, th the summed omegas."""
    X, T = octahedron()
    ratio = 1.1
    o = sim.Simulation.__new__(sim.Simulation)
    o.bodies = []
    o.bodies.append(sim.Body(X, T, dict(rigid=1, density_ratio=ratio), tau=0.8))
    b = o.bodies[0]
    V0 = 4.0 / 3.0
    m = ratio * V0
    r = (3.0 * V0 / (4.0 * math.pi)) ** (1.0 / 3.0)
    inertia = 0.4 * m * r * r
    f = np.array([0.0, 3e-4, 0.0])
    k = 2e-3
    a = f / m
    alpha = 2.0 * k / inertia
    seq = [2.0 / 3.0, 14.0 / 9.0, 68.0 / 27.0]
    centre = np.zeros(3)
    th = 0.0
    for n in range(3):
        F = np.tile(f / 6.0, (6, 1))
        for v in (0, 2):
            rv = b.x[v] - b.xc
            F[v] += k * np.cross([0.0, 0.0, 1.0], rv)
        o.update(None, [{}], [F])
        centre = centre + seq[n] * a
        th += seq[n] * alpha
        np.testing.assert_allclose(b.xc, centre, rtol=0, atol=1e-15)
        np.testing.assert_allclose(b.u1, seq[n] * a, rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(b.w1, [0.0, 0.0, seq[n] * alpha], rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(b.x[0], centre + [math.cos(th), math.sin(th), 0.0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(b.x[1], centre + [-math.sin(th), math.cos(th), 0.0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(b.x[4], centre + [0.0, 0.0, 1.0], rtol=0, atol=1e-14)
        # boundary velocity of the markers: u + omega x r
        wz = seq[n] * alpha
        np.testing.assert_allclose(b.vel[0], seq[n] * a + wz * np.array([-math.sin(th), math.cos(th), 0.0]),
                                   rtol=1e-12, atol=1e-18)
    assert th > 0.05     # the rotation is large enough for a sign error to show


# ---------------------------------------------------------------------------
# Probe stresses (Eqs. hydroForP, hydroForNu; Reading S-d)
# ---------------------------------------------------------------------------
def test_viscous_and_pressure_probe_forces_in_a_linear_field():
    """Populations at equilibrium with a linear density rho = 1 + beta.(x - x0)
    and a linear, non-symmetric velocity gradient u = G (x - x0): the MLS fit
    reproduces both exactly, so at the probes x +- 1.2 n
        tau+ - tau- = 2.4 (beta.n) nu (G + G^T),   p+ - p- = 2.4 (beta.n) / 3,
    and the forces are F_tau = (tau+ - tau-) n A and F_p = -(p+ - p-) n A.  A
    missing transpose, a factor 2, a wrong nu or a swapped probe side fails."""
    n = 16
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    lat = L.Lattice(n, n, n, tau, np.zeros(n ** 3, np.uint8), dict(node=[], dir=[], q=[]), [None] * 6,
                    (False, False, False))
    x0 = np.array([7.3, 8.1, 7.7])
    beta = np.array([2e-3, -1e-3, 1.5e-3])
    Gm = np.array([[0.0, 3e-3, 1e-3], [-1e-3, 5e-4, 0.0], [2e-3, 0.0, -5e-4]])
    P = np.stack([lat.X, lat.Y, lat.Z], axis=1).astype(np.float64) - x0
    rho = 1.0 + P @ beta
    u = P @ Gm.T
    f = lat.init_equilibrium(rho, u)
    rng = np.random.default_rng(4)
    M = 5
    X = x0 + rng.uniform(-1.0, 1.0, (M, 3))
    nrm = rng.standard_normal((M, 3))
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    A = rng.uniform(0.5, 1.5, M)
    Fp, Ft = membrane.hydrodynamic_forces(lat, f, X, A, nrm)
    S = Gm + Gm.T
    for k in range(M):
        bn = 2.4 * float(beta @ nrm[k])
        np.testing.assert_allclose(Ft[k], bn * nu * (S @ nrm[k]) * A[k], rtol=1e-9, atol=1e-18)
        np.testing.assert_allclose(Fp[k], -(bn / 3.0) * nrm[k] * A[k], rtol=1e-9, atol=1e-18)


# ---------------------------------------------------------------------------
# Zou-He faces: mass balance of a steady duct (Eq. extbound)
# ---------------------------------------------------------------------------
def test_zou_he_steady_duct_flux_balance():
    """Poiseuille velocity inlet at x = 0, pressure outlet at x = nx - 1, BFL
    walls: at steady state the mass flux sum(rho u_x) through every
    cross-section, inlet and outlet included, is the same to < 1e-6 relative
    (the geometric approach to steady state is monitored; each 1000 steps cut
    the imbalance about sixfold)."""
    g = G.straight_duct(16, 10, 10, 6.0, u_max=0.02)
    lat = L.Lattice(g.nx, g.ny, g.nz, 1.0, g.tag, g.links, g.faces, g.periodic)
    f = lat.init_equilibrium()
    fl = lat.fluid
    imb = []
    for chunk in range(5):
        for _ in range(1000):
            f = lat.step(f)
        rho, u = lat.macroscopic(f)
        flux = np.array([(rho * u[:, 0])[fl & (lat.X == x)].sum() for x in range(g.nx)])
        imb.append(np.abs(flux - flux.mean()).max() / flux.mean())
    assert flux[0] > 0
    assert imb[-1] < 1e-6, imb
    assert all(b < a for a, b in zip(imb, imb[1:])), imb


# ---------------------------------------------------------------------------
# Duct flow at D = 24
# ---------------------------------------------------------------------------
def test_duct_poiseuille_at_d24():
    """The body-force-driven square duct with walls at q = 0.3 / 0.7: relative
    L2 error against the Fourier-series closed form of 1.75e-3 at D = 24 and
    the same second order from D = 16 to 24 (the error falls by more than
    (24/16)^1.8)."""
    from test_oracle_physics import _duct_run
    e16, _ = _duct_run(16)
    e24, qs = _duct_run(24)
    assert 0.3 in qs and 0.7 in qs
    assert e24 < 2e-3, e24
    assert e16 / e24 > 1.5 ** 1.8, (e16, e24)


# ---------------------------------------------------------------------------
# Reading T1: the structure update takes the fluid solution at t
# ---------------------------------------------------------------------------
def _second_differences(post_collision, steps):
    """RMS over the vertices of x(t+1) - 2 x(t) + x(t-1) every 20 steps for a
    soft capsule (d = 10, 642 v, Ca = 0.05) in a duct at Re = u_max D / nu =
    12, with the step order of Reading T1 or, when post_collision is set,
    with u_v,0 and the probes taken from the populations after the
    collision and stream of the same step."""
    from oracle import ib
    from paper_2207_06043_gb300 import meshes as Ms

    class PostCollision(sim.Simulation):
        def step(self, n=1):
            for _ in range(n):
                f_ib, per = self.ib_force()
                fnew = self.lat.step(self.f, f_ib)
                for b, p in zip(self.bodies, per):
                    p["U"] = ib.interpolate_velocity(fnew, ib.stencil(self.lat, b.x))
                self.update(fnew, per, self.structure(fnew, per))
                self.f = fnew
                self.t += 1
            return n

    u_max, D = 0.06, 20.0
    g = G.straight_duct(40, 24, 24, D, u_max=u_max)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic)
    o = (PostCollision if post_collision else sim.Simulation)(lat, u_max=u_max)
    V, T = Ms.sphere_mesh(642, 10.0, (8.0, g.info["yc"] + 0.7, g.info["zc"]), Ms.SplitMix64(5))
    o.add_body(V, T, dict(Ca=0.05, Eb=0.001, kv=1.0, density_ratio=1.1, u_ref=u_max))
    xs = [o.bodies[0].x.copy()]
    V0 = membrane.diagnostics(o.bodies[0].x, o.bodies[0].tris)["volume"]
    out = []
    for it in range(1, steps + 1):
        o.step(1)
        xs = (xs + [o.bodies[0].x.copy()])[-3:]
        if it % 20 == 0:
            d2 = xs[2] - 2.0 * xs[1] + xs[0]
            out.append(float(np.sqrt((d2 * d2).sum(axis=1).mean())))
    V = membrane.diagnostics(o.bodies[0].x, o.bodies[0].tris)["volume"]
    return np.array(out), V / V0 - 1.0


def test_step_order_reading_t1_keeps_the_membrane_free_of_a_period_two_mode():
    """Reading T1 (the paper does not state the order): the tentative velocity
    u_v,0 of Eq. verletPos and the probe stresses come from the fluid at t,
    the field the IB pre-pass interpolates.  Taking them from the field after
    the collision and stream instead makes the explicit coupling grow a
    period-2 oscillation of the vertices: their second time difference grows
    by orders of magnitude within 160 steps, while with Reading T1 it decays
    from the start-up transient and stays small.  With Reading T1 the capsule
    also keeps its volume within 1 % (volume penalty, Eq. volFor)."""
    t1, dV = _second_differences(False, 160)
    post, _ = _second_differences(True, 160)
    assert t1[-1] < 1e-3 and t1[-4:].max() < t1[0], t1
    assert abs(dV) < 0.01, dV
    assert post[-1] > 30.0 * post[0] and np.all(np.diff(post[1:]) > 0), post


# ---------------------------------------------------------------------------
# Drag of a fixed sphere (Stokes with Hasimoto's periodic-array correction)
# ---------------------------------------------------------------------------
def hasimoto_K(c):
    """Drag factor of a simple cubic array of spheres at volume fraction c
    (Hasimoto's series with the Sangani-Acrivos terms): F = 6 pi mu a U / K."""
    return 1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2 + 3.9799 * c ** (8 / 3) - 3.0734 * c ** (10 / 3)


def test_fixed_sphere_drag_matches_stokes_with_hasimoto_correction():
    """A rigid sphere d = 8 (642 v) held in place (mass 1e9 V0) in a 24^3
    periodic box, driven by a uniform body force g along x from a uniform
    start near the expected mean velocity.  The box-mean flow relaxes on
    L^3 / (drag per unit velocity), about 600 steps, but the flow around the
    sphere is quasi-steady after a few hundred: the drag D = -sum f_ib per
    unit box-mean velocity U then holds to 0.3 % and lies 0 to 15 % above
    Stokes' 6 pi mu a / K(c), the band of an effective hydrodynamic radius
    from a to about a + 0.45 lu for this diffuse interface.  A missing
    c_l = A_l, a wrong sign of F_l or a wrong spreading weight misses it by
    far more."""
    Lb, d, tau, g = 24, 8.0, 1.0, 1e-6
    from paper_2207_06043_gb300 import meshes as Ms
    geo = G.periodic_box(Lb, Lb, Lb)
    lat = L.Lattice(geo.nx, geo.ny, geo.nz, tau, geo.tag, geo.links, geo.faces, geo.periodic,
                    body_force=(g, 0.0, 0.0))
    nu = (tau - 0.5) / 3.0
    a = d / 2
    c = 4.0 / 3.0 * math.pi * a ** 3 / Lb ** 3
    coef = 6 * math.pi * nu * a / hasimoto_K(c)
    u0 = np.zeros((lat.N, 3))
    u0[:, 0] = g * Lb ** 3 / coef / 1.08
    o = sim.Simulation(lat, f0=lat.init_equilibrium(None, u0), u_max=0.02)
    c0 = (Lb - 1) / 2
    V, T = Ms.sphere_mesh(642, d, (c0 + 0.1, c0 + 0.2, c0 + 0.3), Ms.SplitMix64(11))
    o.add_body(V, T, dict(rigid=1, density_ratio=1e9))
    ratios = []
    for _ in range(5):
        o.step(100)
        _, u = lat.macroscopic(o.f)
        D = -o.last["f_ib"].sum(axis=0)
        ratios.append(D[0] / u[:, 0].mean() / coef)
        assert abs(D[1]) < 1e-3 * D[0] and abs(D[2]) < 1e-3 * D[0]
    assert abs(ratios[-1] - ratios[-2]) < 3e-3 * ratios[-1], ratios
    assert 1.0 < ratios[-1] < 1.15, ratios
    assert abs(o.bodies[0].xc[0] - (c0 + 0.1)) < 1e-6


# ---------------------------------------------------------------------------
# Explicit stability of the membrane update (Eqs. verletPos .. verletPosC)
# ---------------------------------------------------------------------------
def _stiffness_kappa(rest, X0, iters=120):
    """lambda_max of the Hessian of the stretch + bend energy at rest, over the
    vertex mass (power iteration on central differences of the forces)."""
    rng = np.random.default_rng(0)
    v = rng.standard_normal(X0.shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        h = 1e-6
        Fp = membrane.stretch_forces(X0 + h * v, rest) + membrane.bending_forces(X0 + h * v, rest)
        Fm = membrane.stretch_forces(X0 - h * v, rest) + membrane.bending_forces(X0 - h * v, rest)
        Hv = -(Fp - Fm) / (2 * h)
        lam = float((v * Hv).sum())
        v = Hv / np.linalg.norm(Hv)
    return lam / rest.mv


def test_membrane_update_is_stable_below_kappa_0_8():
    """Without fluid (u_v,0 = 0) the Verlet update of Eqs. verletPos ..
    verletPosC is x' = (1/2 - 5/4 kappa) x + x_prev / 2 for a mode of
    stiffness lambda over the vertex mass, kappa = lambda / m_v: its roots
    leave the unit circle through -1 at kappa = 4/5.  A perturbed capsule at
    kappa_max = 0.7 stays bounded over 400 steps and one at 0.9 grows by
    orders of magnitude (Ca chosen from the measured kappa_max, which scales
    as 1/Ca)."""
    from paper_2207_06043_gb300 import meshes as Ms
    X0, T = Ms.sphere_mesh(162, 8.0, (0.0, 0.0, 0.0), Ms.SplitMix64(2))
    base = membrane.CapsuleRest(X0, T, dict(Ca=0.01, Eb=0.001, kv=0.0), 0.8)
    k_base = _stiffness_kappa(base, X0)
    amp = {}
    for target in (0.7, 0.9):
        rest = membrane.CapsuleRest(X0, T, dict(Ca=0.01 * k_base / target, Eb=0.001, kv=0.0), 0.8)
        rng = np.random.default_rng(1)
        x = X0 + 1e-4 * rng.standard_normal(X0.shape)
        xp = x.copy()
        for _ in range(400):
            F = membrane.stretch_forces(x, rest) + membrane.bending_forces(x, rest)
            x_new, _ = sim.verlet(x, xp, np.zeros_like(x), F, rest.mv)
            xp, x = x, x_new
        amp[target] = float(np.abs(x - X0 - (x - X0).mean(axis=0)).max())
    assert amp[0.7] < 1e-3, amp
    assert amp[0.9] > 1e2 * amp[0.7], amp


# ---------------------------------------------------------------------------
# Free rigid sphere in quiescent fluid (Section "Rigid structures transport",
# Eq. angularVelRig, with the probe stresses of Eqs. hydroForP, hydroForNu)
# ---------------------------------------------------------------------------
def _free_sphere_momenta(steps_marks, flip_hydro=False, monkeypatch=None):
    from paper_2207_06043_gb300 import meshes as Ms
    if flip_hydro:
        orig = membrane.hydrodynamic_forces
        monkeypatch.setattr(membrane, "hydrodynamic_forces", lambda *a, **k: tuple(-x for x in orig(*a, **k)))
    g = G.periodic_box(20, 20, 20)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic)
    o = sim.Simulation(lat, u_max=0.01)
    V, T = Ms.sphere_mesh(162, 8.0, (10.0, 10.2, 9.9), Ms.SplitMix64(4))
    vel0 = np.array([0.005, 0.001, 0.0])
    o.add_body(V, T, dict(rigid=1, density_ratio=1.1), vel0=vel0)
    b = o.bodies[0]
    out, done = [], 0
    for n in steps_marks:
        o.step(n - done)
        done = n
        fluid = np.einsum("kn,ka->a", o.f, L.Ef)      # sum_i f_i e_i over every node
        out.append((fluid, b.rest.mass * b.u1.copy(), b.u1.copy()))
    return vel0, out


def test_free_rigid_sphere_keeps_its_total_momentum_after_the_start_up(monkeypatch):
    """A rigid sphere (d = 8, density ratio 1.1) released at u0 in fluid at
    rest, periodic box.  The direct forcing drags the fluid inside and around
    the sphere to the sphere's velocity within the first steps, and the
    sphere's own force is the probe traction, not the reaction to that forcing,
    so the start-up adds momentum (here 1.42 -> 3.60 in 20 steps).  After it
    the exchange balances: the sphere slows down, the fluid takes up what it
    loses, the total stays within 5 % over 100 steps (3.6 % measured) and along
    u0.  With the sign of the probe forces on the sphere reversed, the sphere
    is pushed along its motion and the total keeps growing (2.7 times from
    step 20 to step 60, 33 times its value at release)."""
    marks = (20, 60, 120)
    vel0, res = _free_sphere_momenta(marks)
    tot = [f + p for f, p, _ in res]
    drift = np.linalg.norm(tot[-1] - tot[0]) / np.linalg.norm(tot[0])
    assert drift < 0.05, drift
    speeds = [np.linalg.norm(u) for _, _, u in res]
    assert speeds[0] > speeds[1] > speeds[2] > 0, speeds          # the drag slows the sphere
    assert res[2][0] @ vel0 > res[0][0] @ vel0 > 0                   # the fluid takes the momentum up
    cosang = tot[-1] @ vel0 / (np.linalg.norm(tot[-1]) * np.linalg.norm(vel0))
    assert cosang > 1 - 1e-6, cosang                                  # along u0, no cross-stream drift
    # a planted sign error in the sphere's hydrodynamic force
    _, bad = _free_sphere_momenta((20, 60), flip_hydro=True, monkeypatch=monkeypatch)
    grow = np.linalg.norm(bad[1][0] + bad[1][1]) / np.linalg.norm(bad[0][0] + bad[0][1])
    assert grow > 2.0, grow
