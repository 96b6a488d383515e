"""Pins of the oracle's immersed-boundary transfer, membrane mechanics,
structure updates and capsule diagnostics (no GPU)."""
import math

import numpy as np
import pytest

from oracle import ib, lattice as L, membrane as Mb, sim
from paper_2207_06043_gb300 import geometry as G, meshes


def _box_lattice(n=12, periodic=True):
    g = G.periodic_box(n, n, n)
    per = (periodic,) * 3
    return L.Lattice(n, n, n, 0.8, g.tag, g.links, g.faces, per)


# -- MLS ---------------------------------------------------------------------

def test_weight_function_values():
    assert ib.weight_function(np.array([0.0]))[0] == 1.0
    assert ib.weight_function(np.array([1.0]))[0] == pytest.approx(math.exp(-1 / 0.09))
    assert ib.weight_function(np.array([1.0 + 1e-12]))[0] == 0.0


def test_mls_partition_of_unity_and_linear_reproduction():
    lat = _box_lattice()
    rng = np.random.default_rng(1)
    X = rng.uniform(1.0, 10.0, (200, 3))
    st = ib.stencil(lat, X)
    pos = np.stack([lat.X, lat.Y, lat.Z], axis=1).astype(float)[st.nodes]
    assert np.allclose(st.phi.sum(1), 1.0, atol=1e-13)
    assert np.allclose(np.einsum("mk,mkc->mc", st.phi, pos), X, atol=1e-12)
    # gradient weights: derivative of a linear field is exact
    assert np.allclose(st.grad.sum(2), 0.0, atol=1e-12)
    Gm = np.einsum("mjk,mkc->mcj", st.grad, pos)
    assert np.allclose(Gm, np.broadcast_to(np.eye(3), Gm.shape), atol=1e-12)
    # 27 support nodes, all with r <= 1 (support side 2.6 covers the 3x3x3 block)
    assert st.nodes.shape == (200, 27) and (st.weight > 0).all()


def test_mls_near_walls_keeps_solid_nodes_as_wall_data():
    """Reading M4: near a wall every point of the 3x3x3 support takes part,
    the solid ones with the wall's rest state, so the fit keeps the bulk
    weights (partition of unity, linear reproduction, no fallback), and the
    velocity interpolated from a uniform flow U0 in the fluid is U0 times the
    weight of the fluid points alone."""
    g = G.straight_duct(10, 14, 14, 9.0, periodic_x=True)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic)
    rng = np.random.default_rng(2)
    yc = g.info["yc"]
    X = np.stack([rng.uniform(0, 10, 100), yc + rng.uniform(3.0, 4.4, 100), yc + rng.uniform(-4, 4, 100)], 1)
    st = ib.stencil(lat, X)
    solid = ~lat.fluid[st.nodes]
    assert solid.any(axis=1).sum() > 50              # most points see the wall
    assert (st.weight > 0).all() and not st.fallback.any()
    pos = np.stack([lat.X, lat.Y, lat.Z], axis=1).astype(float)[st.nodes]
    assert np.allclose(st.phi.sum(1), 1.0, atol=1e-12)
    # periodic x: unwrap node coordinates near the seam before checking x
    dx = (pos[..., 0] - X[:, None, 0] + 5) % 10 - 5
    assert np.allclose(np.einsum("mk,mk->m", st.phi, dx), 0.0, atol=1e-11)
    assert np.allclose(np.einsum("mk,mk->m", st.phi, pos[..., 1]), X[:, 1], atol=1e-11)
    U0 = np.array([0.02, -0.01, 0.005])
    u = np.where(lat.fluid[:, None], U0[None, :], 0.0)
    f = lat.init_equilibrium(None, u)
    f[:, ~lat.fluid] = L.W[:, None]          # solid nodes: the rest state
    U = ib.interpolate_velocity(f, st)
    w_fluid = np.where(solid, 0.0, st.phi).sum(axis=1)
    assert np.allclose(U, w_fluid[:, None] * U0[None, :], atol=1e-12)
    assert (np.abs(w_fluid - 1.0) > 1e-3).sum() > 20


def test_mls_support_off_the_box_takes_the_nearest_box_node():
    """A point beyond a non-periodic box face keeps its full support; the
    points off the box take the state of the nearest box node (Reading M4),
    so the fit stays regular, and a field that does not vary across the face
    is reproduced exactly."""
    n = 7
    tag = np.zeros(n ** 3, np.uint8)
    lat = L.Lattice(n, n, n, 0.8, tag, np.zeros(0, G.LINK_DTYPE), [G.Face() for _ in range(6)],
                    (False, True, True))
    X = np.array([[-0.8, 3.2, 2.9], [0.3, 4.4, 2.1], [6.4, 3.0, 3.5]])   # y, z clear of the periodic seam
    st = ib.stencil(lat, X)
    assert not st.fallback.any() and (st.weight > 0).all()
    base = np.floor(X + 0.5).astype(int)
    cx = np.clip(base[:, None, 0] + ib.OFFSETS[None, :, 0], 0, n - 1)
    assert np.array_equal(st.nodes % n, cx)
    assert np.allclose(st.phi.sum(axis=1), 1.0, atol=1e-12)
    # a field linear in y and z only, constant in x: reproduced exactly
    u = np.zeros((n ** 3, 3))
    idx = np.arange(n ** 3)
    u[:, 0] = 0.01 * (idx // n % n) - 0.02 * (idx // (n * n))
    f = lat.init_equilibrium(None, u)
    U = ib.interpolate_velocity(f, st)
    # periodic y, z: unwrap the support coordinates relative to the point
    Y = st.nodes // n % n
    Z = st.nodes // (n * n)
    dy = (Y - X[:, None, 1] + n / 2) % n - n / 2
    dz = (Z - X[:, None, 2] + n / 2) % n - n / 2
    want = np.einsum("mk,mk->m", st.phi, 0.01 * (X[:, None, 1] + dy) - 0.02 * (X[:, None, 2] + dz))
    assert np.allclose(U[:, 0], want, atol=1e-12)


def test_spreading_conserves_total_force_and_is_the_transpose_of_interpolation():
    lat = _box_lattice()
    rng = np.random.default_rng(4)
    X = rng.uniform(1.0, 10.0, (60, 3))
    F = rng.standard_normal((60, 3))
    c = rng.uniform(0.3, 1.2, 60)
    st = ib.stencil(lat, X)
    fib = ib.spread(lat.N, st, F, c)
    assert np.allclose(fib.sum(0), (c[:, None] * F).sum(0), atol=1e-12)
    u = rng.standard_normal((lat.N, 3))
    lhs = np.sum(c[:, None] * F * st.interp(u))
    rhs = np.sum(u * fib)
    assert lhs == pytest.approx(rhs, rel=1e-12)


# -- membrane ------------------------------------------------------------------

def _perturbed_capsule(nv=162, seed=0, amp=0.05, params=None):
    X0, T = meshes.sphere_mesh(nv, 8.0, (0, 0, 0))
    params = params or dict(Ca=0.05, Eb=0.01, kv=1.0, u_ref=0.02)
    rest = Mb.CapsuleRest(X0, T, params, 0.8)
    rng = np.random.default_rng(seed)
    X = X0 * np.array([1.1, 0.95, 1.0]) + amp * rng.standard_normal(X0.shape)
    return X0, X, T, rest


def test_rest_dihedral_angles_are_convex():
    X0, _, T, rest = _perturbed_capsule()
    assert (rest.theta0 > 0).all()
    assert rest.topo.edge.shape[0] == 3 * X0.shape[0] - 6


def _fd_grad(energy, X, h=1e-6):
    g = np.zeros_like(X)
    for i in range(X.shape[0]):
        for a in range(3):
            Xp = X.copy(); Xp[i, a] += h
            Xm = X.copy(); Xm[i, a] -= h
            g[i, a] = (energy(Xp) - energy(Xm)) / (2 * h)
    return g


def test_stretch_force_is_minus_energy_gradient():
    _, X, _, rest = _perturbed_capsule(42)
    F = Mb.stretch_forces(X, rest)
    g = _fd_grad(lambda Y: Mb.stretch_energy(Y, rest), X)
    assert np.allclose(F, -g, rtol=1e-6, atol=1e-9 * np.abs(g).max())


def test_bending_force_is_minus_energy_gradient():
    _, X, _, rest = _perturbed_capsule(42, amp=0.2)
    F = Mb.bending_forces(X, rest)
    g = _fd_grad(lambda Y: Mb.bending_energy(Y, rest), X)
    assert np.abs(g).max() > 0
    assert np.allclose(F, -g, rtol=1e-6, atol=1e-8 * np.abs(g).max())


def test_internal_forces_have_no_net_force_or_torque():
    _, X, _, rest = _perturbed_capsule(162, amp=0.1)
    for F in (Mb.stretch_forces(X, rest), Mb.bending_forces(X, rest)):
        scale = np.abs(F).max()
        assert np.allclose(F.sum(0), 0.0, atol=1e-12 * scale * len(F))
        assert np.allclose(np.cross(X, F).sum(0), 0.0, atol=1e-11 * scale * len(F))


def test_rigid_motion_gives_no_internal_force():
    X0, _, T, rest = _perturbed_capsule(162)
    R = sim.rotation_matrix(np.array([0.3, -0.2, 0.5]))
    X = X0 @ R.T + np.array([3.0, -1.0, 2.0])
    assert np.abs(Mb.stretch_forces(X, rest)).max() < 1e-13
    assert np.abs(Mb.bending_forces(X, rest)).max() < 1e-13


def test_volume_force_restores_volume():
    X0, _, T, rest = _perturbed_capsule(162)
    for s in (0.97, 1.03):
        X = X0 * s
        d = Mb.diagnostics(X, T)
        Av, nrm = Mb.vertex_areas_normals(X, T, X.shape[0])
        F = Mb.volume_forces(X, rest, d["volume"], Av, nrm)
        radial = np.einsum("ij,ij->i", F, X / np.linalg.norm(X, axis=1)[:, None])
        assert (np.sign(radial) == (1 if s < 1 else -1)).all()


# -- diagnostics -----------------------------------------------------------------

def _box_mesh(a, b, c, centre):
    V = np.array([[x, y, z] for z in (-0.5, 0.5) for y in (-0.5, 0.5) for x in (-0.5, 0.5)])
    V = V * np.array([a, b, c]) + centre
    quads = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    T = []
    for q in quads:
        T += [(q[0], q[1], q[2]), (q[0], q[2], q[3])]
    return V, np.array(T)


def test_diagnostics_exact_on_a_box():
    a, b, c = 3.0, 2.0, 5.0
    ctr = np.array([1.5, -2.0, 0.7])
    V, T = _box_mesh(a, b, c, ctr)
    d = Mb.diagnostics(V, T)
    assert d["volume"] == pytest.approx(a * b * c, rel=1e-14)
    assert d["area"] == pytest.approx(2 * (a * b + b * c + a * c), rel=1e-14)
    assert np.allclose(d["centroid"], ctr, atol=1e-13)
    assert np.allclose(d["second_moment"], np.diag([a * a, b * b, c * c]) * a * b * c / 12, atol=1e-12)


def test_taylor_deformation_of_sphere_and_ellipsoid():
    X, T = meshes.sphere_mesh(2562, 20.0, (3, 4, 5))
    d = Mb.diagnostics(X, T)
    assert d["taylor_D"] < 1e-3
    assert d["volume"] == pytest.approx(4 / 3 * math.pi * 1000, rel=5e-3)
    X, T = meshes.ellipsoid_mesh(2562, (12.0, 9.0, 7.0), (0, 0, 0))
    d = Mb.diagnostics(X, T)
    assert d["taylor_D"] == pytest.approx((12 - 7) / (12 + 7), rel=5e-3)


# -- structure updates -----------------------------------------------------------

def test_verlet_hand_computed_sequence():
    """m_v = 2, F = 0.4 x, u_v0 = 0.1 x, start at rest at 0:
    x = 0.4, 0.6, 0.9 and u = 0.3, 0.1, 0.2 by hand from Eqs. verletPos-verletPosC."""
    x = np.zeros((1, 3)); xp = np.zeros((1, 3))
    F = np.array([[0.4, 0, 0]]); uv0 = np.array([[0.1, 0, 0]])
    xs, us = [], []
    for _ in range(3):
        xn, un = sim.verlet(x, xp, uv0, F, 2.0)
        xp, x = x, xn
        xs.append(xn[0, 0]); us.append(un[0, 0])
    assert np.allclose(xs, [0.4, 0.6, 0.9], atol=1e-15)
    assert np.allclose(us, [0.3, 0.1, 0.2], atol=1e-15)


def test_rigid_velocity_rule():
    assert sim.rigid_velocity(1.0, 0.5, 0.3) == pytest.approx(2.0 / 3.0 * 2.05, abs=1e-15)
    # steady state is a fixed point
    assert sim.rigid_velocity(0.7, 0.7, 0.0) == pytest.approx(0.7, abs=1e-15)


def test_repulsion_magnitude_and_direction():
    Xa = np.array([[0.0, 0.0, 0.0]]); na = np.array([[1.0, 0.0, 0.0]])
    Xb = np.array([[1.0, 0.0, 0.0]]); nb = np.array([[-1.0, 0.0, 0.0]])
    Fa, Fb = Mb.repulsion_forces([Xa, Xb], [na, nb], 0.02)
    w = 0.02 / (8 * math.sqrt(2))
    assert np.allclose(Fa, [[-w, 0, 0]]) and np.allclose(Fb, [[w, 0, 0]])
    Xb2 = np.array([[2.5, 0.0, 0.0]])
    Fa, _ = Mb.repulsion_forces([Xa, Xb2], [na, nb], 0.02)
    assert np.all(Fa == 0)


def test_hydrodynamic_pressure_force_from_linear_density():
    """With rho = 1 + beta x at rest the MLS probes see p+ - p- = beta/3 * 2.4 n_x
    exactly, and the viscous term vanishes."""
    n = 20
    g = G.periodic_box(n, n, n)
    lat = L.Lattice(n, n, n, 0.8, g.tag, g.links, g.faces, (False,) * 3)
    beta = 1e-3
    rho = 1 + beta * lat.X
    f = lat.init_equilibrium(rho, None)
    X, T = meshes.sphere_mesh(162, 6.0, (10, 10, 10))
    Av, nrm = Mb.vertex_areas_normals(X, T, X.shape[0])
    Fp, Ft = Mb.hydrodynamic_forces(lat, f, X, Av, nrm)
    exp = -(beta / 3.0 * 2.4 * nrm[:, 0] * Av)[:, None] * nrm
    assert np.allclose(Fp, exp, atol=1e-14)
    assert np.abs(Ft).max() < 1e-14


# -- damage rule (Section "Transport of an elastic capsule") ---------------------

def test_largest_stretch_of_a_scaled_mesh_is_the_scale_and_two_stops_the_run():
    """Every edge of a mesh scaled by s about any point is s times its rest
    length, so the largest stretch is s (to rounding); an edge at twice its
    rest length is the damage of the paper's rule and stops the run at the
    step that finds it (the lattice is not stepped further)."""
    X, T = meshes.sphere_mesh(162, 8.0, (6.0, 6.0, 6.0), meshes.SplitMix64(3))
    rest = Mb.CapsuleRest(X, T, dict(Ca=0.05), 0.8)
    c = X.mean(axis=0)
    for s in (1.0, 1.25, 1.999):
        assert abs(Mb.max_stretch(c + s * (X - c), rest) - s) < 1e-12, s
    lat = _box_lattice(12)
    o = sim.Simulation(lat, u_max=0.01)
    o.add_body(X, T, dict(Ca=0.05))
    assert o.step(1) == 1 and not o.damaged
    o.bodies[0].x = c + 2.0 * (o.bodies[0].x - c)
    o.bodies[0].x_prev = o.bodies[0].x.copy()
    assert o.step(3) == 1 and o.damaged          # found at the end of that step
    assert o.step(5) == 0                         # nothing more runs
