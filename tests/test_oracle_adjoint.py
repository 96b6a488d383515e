"""Pins of the oracle's discrete adjoint (CPU): each transposed operator
against its forward operator on random vectors (dot-product test), and the
whole reverse sweep against central finite differences of the objective."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import lattice as L
from paper_2207_06043_gb300 import geometry as G


@pytest.fixture(scope="module")
def setup():
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.02, with_dq=True)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic)
    f = lat.init_equilibrium()
    for _ in range(25):
        f = lat.step(f)
    dq = g.links["dq"].astype(np.float64)
    return g, lat, f, dq


def _rand(lat, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((19, lat.N))


def test_geometry_carries_link_sensitivities(setup):
    g, lat, f, dq = setup
    assert np.count_nonzero(dq) > 100          # links on the fillet move with r_j
    assert np.isfinite(dq).all()


def test_stream_transpose(setup):
    _, lat, _, _ = setup
    lam, dl = _rand(lat, 1), _rand(lat, 2)
    lhs = np.nansum(lam * lat.stream(dl))
    rhs = (A.stream_vjp(lat, lam) * dl).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_wall_link_transpose(setup):
    _, lat, f, dq = setup
    lam, dl = _rand(lat, 3), _rand(lat, 4)
    xb, i, ib, *_ = lat.link_neighbours()
    out = np.full((19, lat.N), np.nan)
    lat.bouzidi(out, dl)                         # the link rule is linear in f*
    lhs = (lam[ib, xb] * out[ib, xb]).sum()
    lam_only = np.zeros_like(lam)
    lam_only[ib, xb] = lam[ib, xb]
    adj, _ = A.bfl_vjp(lat, lam_only, dl, dq)
    rhs = (adj * dl).sum()
    assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_face_rule_transpose(setup):
    _, lat, f, _ = setup
    fstar = lat.collide_all(f, None)
    fb = lat.bouzidi(lat.stream(fstar), fstar)
    base = np.nan_to_num(fb)
    nodes = np.concatenate([lat.face_nodes(k)[0] for k, s in enumerate(lat.faces) if s is not None and s.kind])
    lam, dl = _rand(lat, 5), 1e-3 * _rand(lat, 6)
    z0 = lat.zou_he(base.copy())
    z1 = lat.zou_he(base + dl)
    lhs = (lam[:, nodes] * (z1 - z0)[:, nodes]).sum()    # the face rule is affine in f
    adj, _ = A.zh_vjp(lat, lam, fb)
    rhs = (adj[:, nodes] * dl[:, nodes]).sum()
    assert abs(lhs - rhs) <= 1e-9 * abs(lhs)


def test_collision_transpose_against_finite_differences(setup):
    _, lat, f, _ = setup
    lam, dl = _rand(lat, 7), _rand(lat, 8)
    h = 1e-6
    jvp = (lat.collide_all(f + h * dl, None) - lat.collide_all(f - h * dl, None)) / (2 * h)
    fl = lat.fluid
    lhs = (lam[:, fl] * jvp[:, fl]).sum()
    rhs = (A.collide_vjp(lat, f, lam)[:, fl] * dl[:, fl]).sum()
    assert abs(lhs - rhs) <= 1e-7 * abs(lhs)


def test_adjoint_gradient_matches_central_differences(setup):
    """dJ/ds_u (inlet velocity scale) and dJ/ds_q (link distances moved along
    dq/dr_j) over 12 steps against central differences with h = 1e-4."""
    g, lat, f, dq = setup
    obj = A.Objective(lo=(2, 0, 0), hi=(24, 20, 16), d=(1.0, 0.3, 0.0))
    steps = 12
    J, gu, gq = A.gradient(lat, f, steps, obj, dq)
    assert J == pytest.approx(A.value(lat, f, steps, obj), rel=1e-13)
    h = 1e-4
    fd_u = (A.value(A.perturbed(lat, s_u=h), f, steps, obj)
            - A.value(A.perturbed(lat, s_u=-h), f, steps, obj)) / (2 * h)
    fd_q = (A.value(A.perturbed(lat, s_q=h, dq=dq), f, steps, obj)
            - A.value(A.perturbed(lat, s_q=-h, dq=dq), f, steps, obj)) / (2 * h)
    assert gu == pytest.approx(fd_u, rel=1e-6)
    assert gq == pytest.approx(fd_q, rel=1e-6)
    assert abs(gu) > 1e-6 and abs(gq) > 1e-9


def _capsule_case():
    from paper_2207_06043_gb300 import meshes as Ms
    from paper_2207_06043_gb300 import workloads as W
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.03, with_dq=True)
    V, T = Ms.sphere_mesh(162, 7.0, (9.0, g.info["yc"] + 0.4, g.info["zc"] - 0.3), Ms.SplitMix64(4))
    return dict(geometry=g, tau=0.8, u_max=0.03, capsules=[W._capsule(V, T, Ca=0.05, u_ref=0.03)])


def test_coupled_capsule_derivative_matches_central_differences():
    """The derivative of J = D + 0.5 (y_c - y_sym) of a soft capsule after 30
    coupled steps (IB, membrane, probes, Verlet, lattice with BFL and Zou-He)
    with respect to Ca, u_max and the junction radius, taken by the complex
    step through the whole oracle run, against central differences of the
    oracle with h = 1e-4 relative: agreement to 1e-6 relative."""
    c = _capsule_case()
    steps, yc = 30, c["geometry"].info["yc"]
    J, g_ca, g_um, g_rj = A.coupled_gradient(c, steps, 1.0, 0.5, yc)
    for kw, p, g, scale in (("dCa", 0.05, g_ca, 1.0), ("ds_u", 1.0, g_um, 1.0 / 0.03), ("ds_q", 1.0, g_rj, 1.0)):
        h = 1e-4 * p
        jp = A.coupled_run(c, steps, 1.0, 0.5, yc, **{kw: h})[0]
        jm = A.coupled_run(c, steps, 1.0, 0.5, yc, **{kw: -h})[0]
        fd = (jp - jm) / (2 * h) * scale
        assert abs(fd - g) <= 1e-6 * abs(g), (kw, fd, g)
    assert g_ca != 0.0 and g_um != 0.0 and g_rj != 0.0
