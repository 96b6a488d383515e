"""Pins of the FP64 oracle's lattice part against what the paper and the
mathematics fix (no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import lattice as L
from paper_2207_06043_gb300 import geometry as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=7):
    return np.random.default_rng(seed)


# -- velocity set ------------------------------------------------------------

def test_velocity_set_matches_printed_matrix():
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLD, "d3q19_velocities.txt"))
            if l.strip() and not l.startswith("#")]
    assert np.array_equal(np.array(rows).T, L.E)


def test_weights_isotropy_and_opposites():
    E, W = L.Ef, L.W
    assert math.isclose(W.sum(), 1.0, abs_tol=1e-15)
    assert np.allclose(W @ E, 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", W, E, E), L.CS2 * np.eye(3), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", W, E, E, E), 0.0, atol=1e-16)
    d = np.eye(3)
    iso4 = L.CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                         + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", W, E, E, E, E), iso4, atol=1e-16)
    assert np.array_equal(L.E[L.OPP], -L.E)
    assert L.OPP[0] == 0 and np.array_equal(L.OPP[L.OPP], np.arange(19))


# -- equilibrium and forcing moments ------------------------------------------

def test_equilibrium_moments():
    r = _rng()
    n = 50
    rho = 1.0 + 0.1 * r.standard_normal(n)
    u = 0.05 * r.standard_normal((n, 3))
    feq = L.equilibrium(rho, u)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    assert np.allclose((L.Ef.T @ feq).T, rho[:, None] * u, atol=1e-15)
    Pi = np.einsum("in,ia,ib->nab", feq, L.Ef, L.Ef)
    ref = rho[:, None, None] * (L.CS2 * np.eye(3)[None] + np.einsum("na,nb->nab", u, u))
    assert np.allclose(Pi, ref, atol=1e-14)


def test_guo_forcing_moments():
    r = _rng(3)
    n = 40
    tau = 0.8
    u = 0.05 * r.standard_normal((n, 3))
    F = 1e-3 * r.standard_normal((n, 3))
    Fi = L.guo_forcing(u, F, tau)
    c = 1.0 - 0.5 / tau
    assert np.allclose(Fi.sum(0), 0.0, atol=1e-18)
    assert np.allclose((L.Ef.T @ Fi).T, c * F, atol=1e-18)
    P = np.einsum("in,ia,ib->nab", Fi, L.Ef, L.Ef)
    ref = c * (np.einsum("na,nb->nab", u, F) + np.einsum("na,nb->nab", F, u))
    assert np.allclose(P, ref, atol=1e-18)


def test_collision_conserves_mass_and_adds_force():
    r = _rng(5)
    n = 30
    f = L.equilibrium(1 + 0.05 * r.standard_normal(n), 0.03 * r.standard_normal((n, 3)))
    f += 1e-3 * r.standard_normal(f.shape)
    F = 1e-3 * r.standard_normal((n, 3))
    fs = L.collide(f, F, 0.7)
    assert np.allclose(fs.sum(0), f.sum(0), atol=1e-15)
    assert np.allclose((L.Ef.T @ fs).T, (L.Ef.T @ f).T + F, atol=1e-15)


# -- whole steps in a periodic box ---------------------------------------------

def test_periodic_box_mass_and_momentum():
    g = G.periodic_box(6, 5, 4)
    F = np.array([1e-5, -2e-5, 3e-6])
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.9, g.tag, g.links, g.faces, g.periodic, body_force=F)
    r = _rng(11)
    f = lat.init_equilibrium(1 + 0.01 * r.standard_normal(lat.N), 0.01 * r.standard_normal((lat.N, 3)))
    m0 = f.sum()
    p0 = (L.Ef.T @ f).sum(axis=1)
    for _ in range(10):
        f = lat.step(f)
    assert abs(f.sum() - m0) < 1e-11
    p = (L.Ef.T @ f).sum(axis=1)
    assert np.allclose(p - p0, 10 * lat.N * F, atol=1e-12)


def test_periodic_box_momentum_gain_equals_a_varying_ib_force():
    """Guo forcing (Eq. forcing) with a force field that differs from node to
    node, as the spread IB force does: mass is kept and every step adds
    exactly sum_k f_ib^k to the momentum (Sigma F_i e_i = (1 - 1/2tau) F plus
    the F/2 carried by the equilibrium through rho u = sum f e + F/2)."""
    g = G.periodic_box(6, 5, 4)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.7, g.tag, g.links, g.faces, g.periodic)
    r = _rng(12)
    f = lat.init_equilibrium(1 + 0.01 * r.standard_normal(lat.N), 0.01 * r.standard_normal((lat.N, 3)))
    m0 = f.sum()
    p = (L.Ef.T @ f).sum(axis=1)
    for s in range(5):
        fib = 1e-4 * r.standard_normal((lat.N, 3))
        f = lat.step(f, fib)
        p_new = (L.Ef.T @ f).sum(axis=1)
        assert np.allclose(p_new - p, fib.sum(axis=0), rtol=0, atol=1e-13), s
        p = p_new
    assert abs(f.sum() - m0) < 1e-11


def test_shear_wave_decay_rate():
    """u_y = U sin(k x) in a periodic box decays as exp(-nu k^2 t), nu = (tau - 1/2)/3."""
    nx = 32
    g = G.periodic_box(nx, 1, 1)
    tau = 0.8
    lat = L.Lattice(nx, 1, 1, tau, g.tag, g.links, g.faces, g.periodic)
    k = 2 * math.pi / nx
    U = 1e-3
    u = np.zeros((nx, 3))
    u[:, 1] = U * np.sin(k * np.arange(nx))
    f = lat.init_equilibrium(None, u)
    steps = 300
    for _ in range(steps):
        f = lat.step(f)
    _, uu = lat.macroscopic(f)
    amp = 2.0 / nx * np.sum(uu[:, 1] * np.sin(k * np.arange(nx)))
    expect = U * math.exp(-L.viscosity(tau) * k * k * steps)
    assert abs(amp / expect - 1.0) < 5e-3


# -- Zou-He ------------------------------------------------------------------

def _face_lattice(face, kind, rng):
    nx, ny, nz = 5, 4, 6
    periodic = [True, True, True]
    periodic[face // 2] = False
    tag = np.zeros(nx * ny * nz, np.uint8)
    faces = [G.Face() for _ in range(6)]
    fs = G.face_shape(face, nx, ny, nz)
    if kind == L.FACE_VELOCITY:
        vel = (0.02 * rng.standard_normal((fs[0] * fs[1], 3))).astype(np.float32)
        faces[face] = G.Face(G.FACE_VELOCITY, 1.0, vel)
    else:
        faces[face] = G.Face(G.FACE_PRESSURE, 1.013, None)
    other = face ^ 1
    faces[other] = G.Face(G.FACE_PRESSURE, 1.0, None)
    links = np.zeros(0, G.LINK_DTYPE)
    return L.Lattice(nx, ny, nz, 0.8, tag, links, faces, periodic)


@pytest.mark.parametrize("face", range(6))
@pytest.mark.parametrize("kind", [L.FACE_VELOCITY, L.FACE_PRESSURE])
def test_zou_he_imposes_the_face_moments(face, kind):
    rng = _rng(100 + face)
    lat = _face_lattice(face, kind, rng)
    nodes, fidx = lat.face_nodes(face)
    f = lat.init_equilibrium(1 + 0.01 * rng.standard_normal(lat.N), 0.02 * rng.standard_normal((lat.N, 3)))
    f += 1e-3 * rng.standard_normal(f.shape)
    nrm = L.FACE_NORMALS[face]
    unknown = np.nonzero(L.E @ nrm < 0)[0]
    f[np.ix_(unknown, nodes)] = np.nan
    lat.zou_he(f)
    sub = f[:, nodes]
    assert not np.isnan(sub).any()
    rho = sub.sum(0)
    mom = (L.Ef.T @ sub).T
    spec = lat.faces[face]
    if kind == L.FACE_VELOCITY:
        uw = spec.velocity[fidx].astype(np.float64)
        assert np.allclose(mom, rho[:, None] * uw, atol=1e-15)
    else:
        assert np.allclose(rho, spec.rho, atol=1e-15)
        tang = [a for a in range(3) if nrm[a] == 0]
        assert np.allclose(mom[:, tang], 0.0, atol=1e-15)


def test_zou_he_reduces_to_printed_north_wall_block():
    """For the z = z_max wall the generic rule equals Eq. extbound as printed,
    with the paper's own labels for that block mapped to velocity vectors
    (Reading Z) and the factor rho on the 1/6 terms (Reading Z')."""
    lab = {}
    for line in open(os.path.join(GOLD, "zou_he_north_wall.txt")):
        if line.strip() and not line.startswith("#"):
            key, *vals = line.split()
            lab[key] = vals
    vec = {0: (0, 0, 0), 1: (1, 0, 0), 2: (-1, 0, 0), 3: (0, 1, 0), 4: (0, -1, 0), 5: (0, 0, 1),
           6: (0, 0, -1), 7: (1, 1, 0), 8: (-1, -1, 0), 9: (1, 0, 1), 10: (-1, 0, -1), 11: (0, 1, 1),
           12: (0, -1, -1), 13: (1, -1, 0), 14: (-1, 1, 0), 15: (1, 0, -1), 16: (-1, 0, 1),
           17: (0, 1, -1), 18: (0, -1, 1)}
    # the label map is consistent with the block's own sets
    assert all(vec[int(a)][2] == 0 for a in lab["rho_zero_sum"])
    assert all(vec[int(a)][2] == 1 for a in lab["rho_known_in"])
    assert all(vec[int(a)][2] == -1 for a in lab["unknown"])
    for pr in lab["pairs"]:
        a, b = map(int, pr.split(":"))
        assert tuple(-np.array(vec[a])) == vec[b]
    to_paper = {lbl: int(np.nonzero((L.E == np.array(v)).all(axis=1))[0][0]) for lbl, v in vec.items()}

    rng = _rng(21)
    lat = _face_lattice(5, L.FACE_VELOCITY, rng)
    nodes, fidx = lat.face_nodes(5)
    f = lat.init_equilibrium(1 + 0.01 * rng.standard_normal(lat.N), 0.02 * rng.standard_normal((lat.N, 3)))
    f += 1e-3 * rng.standard_normal(f.shape)
    uw = lat.faces[5].velocity[fidx].astype(np.float64)
    g = lambda lbl: f[to_paper[lbl], nodes]
    ux, uy, uz = uw[:, 0], uw[:, 1], uw[:, 2]
    rho = (sum(g(int(a)) for a in lab["rho_zero_sum"]) + 2 * sum(g(int(a)) for a in lab["rho_known_in"])) / (uz + 1)
    Nzx = 0.5 * (sum(g(int(a)) for a in lab["Nzx_plus"]) - sum(g(int(a)) for a in lab["Nzx_minus"])) - rho * ux / 3
    Nzy = 0.5 * (sum(g(int(a)) for a in lab["Nzy_plus"]) - sum(g(int(a)) for a in lab["Nzy_minus"])) - rho * uy / 3
    printed = {6: g(5) - rho * uz / 3,
               15: g(16) + rho * (-uz + ux) / 6 - Nzx,
               10: g(9) + rho * (-uz - ux) / 6 + Nzx,
               17: g(18) + rho * (-uz + uy) / 6 - Nzy,
               12: g(11) + rho * (-uz - uy) / 6 + Nzy}
    lat.zou_he(f)
    for lbl, val in printed.items():
        assert np.allclose(f[to_paper[lbl], nodes], val, atol=1e-16)


# -- Bouzidi-Firdaouss-Lallemand ---------------------------------------------------

def _bfl_value(q, fi_b, fi_1, fi_2, fib_b, fib_1):
    """Evaluate the oracle's BFL rule on one synthetic link (all upstream fluid)."""
    nx = 8
    tag = np.zeros(nx, np.uint8)
    tag[nx - 1] = 1
    links = np.zeros(1, G.LINK_DTYPE)
    links[0] = (nx - 2, 1, q, 0.0)
    lat = L.Lattice(nx, 1, 1, 0.8, tag, links, [G.Face() for _ in range(6)], (False, True, True))
    fstar = np.zeros((19, nx))
    xb = nx - 2
    fstar[1, xb], fstar[1, xb - 1], fstar[1, xb - 2] = fi_b, fi_1, fi_2
    fstar[2, xb], fstar[2, xb - 1] = fib_b, fib_1
    fnew = np.zeros((19, nx))
    lat.bouzidi(fnew, fstar)
    return fnew[2, xb]


def test_bfl_halfway_limit_and_weights():
    assert _bfl_value(0.5, 0.3, 0.7, 1.1, 0.2, 0.9) == pytest.approx(0.3, abs=1e-15)
    for q in (0.05, 0.3, 0.49, 0.5, 0.62, 0.99, 1.0):
        # weights sum to one: a uniform field is reproduced
        assert _bfl_value(q, 1.0, 1.0, 1.0, 1.0, 1.0) == pytest.approx(1.0, abs=1e-14)


def test_bfl_reproduces_quadratic_profiles():
    """A population profile quadratic along the link is bounced back exactly:
    the rule is a quadratic Lagrange interpolation (Reading B).  With the wall at
    s = q (s measured along e_i from x_b), the incoming f_ib at s = 0 equals the
    outgoing f_i profile evaluated at the mirror point s = 2q - 1 (q < 1/2), or
    the f_ib profile continued through the reflected point (q >= 1/2)."""
    a, b, c = 0.3, -0.7, 0.45
    prof = lambda s: a + b * s + c * s * s
    for q in (float(np.float32(v)) for v in (0.1, 0.25, 0.4)):
        got = _bfl_value(q, prof(0.0), prof(-1.0), prof(-2.0), 0.0, 0.0)
        assert got == pytest.approx(prof(2 * q - 1), abs=1e-14)
    # q >= 1/2: the returning f_ib is known at s = 2q-1 (value f*_i(x_b)),
    # s = -1 (f*_ib(x_b)) and s = -2 (f*_ib(x_b - e_i)); the rule gives s = 0.
    for q in (float(np.float32(v)) for v in (0.5, 0.7, 0.95)):
        got = _bfl_value(q, prof(2 * q - 1), 0.0, 0.0, prof(-1.0), prof(-2.0))
        assert got == pytest.approx(prof(0.0), abs=1e-14)
