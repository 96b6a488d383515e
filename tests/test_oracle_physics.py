"""Whole-step physics pins of the FP64 oracle: closed-form flows that fix the
collision, the wall rule and its order of accuracy (no GPU)."""
import math

import numpy as np
import pytest

from oracle import lattice as L
from paper_2207_06043_gb300 import geometry as G


def duct_closed_form(y, z, a, b, F, nu, terms=61):
    """Fully developed flow in the rectangular duct |y|<a, |z|<b under a uniform
    body force F (nu lap u = -F): the classical Fourier series."""
    s = np.zeros_like(y)
    for k in range(terms):
        n = 2 * k + 1
        beta = n * math.pi / (2 * a)
        s += (-1) ** k / n ** 3 * (1 - np.cosh(beta * z) / np.cosh(beta * b)) * np.cos(beta * y)
    return 16 * a * a * F / (nu * math.pi ** 3) * s


def _duct_run(D, tau=0.8, steps=None):
    """Square duct, periodic along x (one node), walls offset so that q = 0.3 at
    one wall and 0.7 at the other, driven by a body force along x."""
    n = D + 4
    yc = (n - 1) / 2 + 0.2
    g = G.straight_duct(1, n, n, D, periodic_x=True, centre=(yc, yc))
    F = 1e-6
    lat = L.Lattice(g.nx, g.ny, g.nz, tau, g.tag, g.links, g.faces, g.periodic, body_force=(F, 0, 0))
    nu = L.viscosity(tau)
    lam = 2 * nu * math.pi ** 2 / D ** 2
    steps = steps or int(16.0 / lam)
    f = lat.init_equilibrium()
    for _ in range(steps):
        f = lat.step(f)
    _, u = lat.macroscopic(f)
    fl = lat.fluid
    ue = duct_closed_form(lat.Y[fl] - yc, lat.Z[fl] - yc, D / 2, D / 2, F, nu)
    return np.linalg.norm(u[fl, 0] - ue) / np.linalg.norm(ue), sorted(set(np.round(g.links["q"], 4)))


def test_duct_poiseuille_closed_form_and_order():
    e8, qs = _duct_run(8)
    e16, _ = _duct_run(16)
    assert 0.3 in qs and 0.7 in qs
    assert e16 < 1e-2
    order = math.log(e8 / e16, 2)
    assert order > 1.6, (e8, e16, order)


def _inclined_run(width, tau=1.0):
    g = G.inclined_channel(width)
    F = 1e-6
    ax = g.info["axis"]
    lat = L.Lattice(g.nx, g.ny, g.nz, tau, g.tag, g.links, g.faces, g.periodic, body_force=F * ax)
    nu = L.viscosity(tau)
    P = np.stack([lat.X, lat.Y, lat.Z], axis=1).astype(float)
    s = P @ g.info["normal"] - g.info["centre"]
    per = g.info["period"]
    s = (s + 0.5 * per) % per - 0.5 * per
    uex = F / (2 * nu) * (width ** 2 / 4 - s ** 2)
    u0 = np.where(lat.fluid[:, None], uex[:, None] * ax[None, :], 0.0)
    f = lat.init_equilibrium(None, u0)
    steps = int(8.0 * width ** 2 / (nu * math.pi ** 2))
    for _ in range(steps):
        f = lat.step(f)
    _, u = lat.macroscopic(f)
    fl = lat.fluid
    ua = u[fl] @ ax
    return np.linalg.norm(ua - uex[fl]) / np.linalg.norm(uex[fl])


def test_bfl_second_order_on_inclined_channel():
    """Planar channel inclined at atan(1/2), periodic along the channel: the
    error against the parabola falls as width^-2 (least-squares slope of the
    relative L2 error over widths 8, 16, 24 within 1.8 .. 2.2)."""
    widths = np.array([8.0, 16.0, 24.0])
    e = np.array([_inclined_run(int(w)) for w in widths])
    slope = -np.polyfit(np.log(widths), np.log(e), 1)[0]
    assert 1.8 < slope < 2.2, (e, slope)
