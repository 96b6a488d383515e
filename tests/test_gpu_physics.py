"""Physics of the whole coupled method on the CUDA path (GPU): checks against
closed forms and the paper's qualitative findings that need more steps than
the FP64 oracle can take in a test.  The CUDA path matches the oracle step for
step elsewhere (tests/test_gpu_parity.py); these pin what both compute."""
import math

import numpy as np
import pytest

from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W

from helpers import case, gpu_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def hasimoto_K(c):
    """Drag correction of a simple cubic array of spheres at volume fraction c
    (Hasimoto's series as extended by Sangani and Acrivos):
    F = 6 pi mu a U / K."""
    return 1 - 1.7601 * c ** (1 / 3) + c - 1.5593 * c ** 2 + 3.9799 * c ** (8 / 3) - 3.0734 * c ** (10 / 3)


def test_sphere_drag_in_a_periodic_array_matches_hasimoto():
    """A rigid sphere (d = 16, 2562 v) too heavy to move, in a 64^3 periodic
    box driven by a uniform body force g (Re about 0.06): at steady state the
    drag is g L^3.  Against Stokes drag with Hasimoto's periodic-array
    correction at the box-mean velocity, the ratio lies between 0.97 and 1.12.
    That is the band of an effective hydrodynamic radius between a - 0.25 and
    a + 0.9 lattice units, the known spread of diffuse-interface IB spheres.
    A missing c_l = A_l, a wrong sign of F_l or a wrong spreading weight
    misses it by far more."""
    L, d, tau, g = 64, 16.0, 1.0, 1e-7
    geo = G.periodic_box(L, L, L)
    c0 = (L - 1) / 2
    V, T = Ms.sphere_mesh(2562, d, (c0 + 0.1, c0 + 0.2, c0 + 0.3), Ms.SplitMix64(11))
    s = gpu_for(case(geo, tau=tau, body_force=(g, 0.0, 0.0),
                     capsules=[W._capsule(V, T, rigid=True, density_ratio=1e9)]))
    means = []
    for _ in range(8):                     # the mean flow spins up on about 7000 steps
        s.step(6000)
        _, u = s.read_fields()
        means.append(float(u[:, 0].mean()))
    U = means[-1]
    assert abs(means[-1] - means[-2]) < 2e-3 * abs(U)        # steady
    nu = (tau - 0.5) / 3.0
    a = d / 2
    c = 4.0 / 3.0 * math.pi * a ** 3 / L ** 3
    drag = g * L ** 3
    stokes = 6 * math.pi * nu * a * U / hasimoto_K(c)
    ratio = drag / stokes
    print(f"drag / (Stokes-Hasimoto) = {ratio:.4f} at U = {U:.4e}")
    assert 0.97 < ratio < 1.12, ratio
    assert abs(s.read_capsule(0)["centroid"][0] - (c0 + 0.1)) < 0.05   # held in place


@pytest.mark.parametrize("Ca", [0.03, 0.1])
def test_capsule_volume_is_conserved_in_duct_flow(Ca):
    """A soft capsule (d = 12, 642 v) carried 2000 steps through a duct keeps
    its volume within 1 % (volume penalty, Eq. volFor)."""
    geo = G.straight_duct(96, 28, 28, 24.0, u_max=0.03)
    V, T = Ms.sphere_mesh(642, 12.0, (14.0, geo.info["yc"] + 1.0, geo.info["zc"]), Ms.SplitMix64(5))
    s = gpu_for(case(geo, u_max=0.03, capsules=[W._capsule(V, T, Ca=Ca, u_ref=0.03)]))
    V0 = s.read_capsule(0)["volume"]
    s.step(2000)
    st = s.read_capsule(0)
    assert not st["damaged"]
    assert abs(st["volume"] - V0) / V0 < 0.01
    assert st["centroid"][0] > 14.0 + 5.0      # it moved downstream


def test_softer_capsules_deform_more():
    """Taylor deformation after 1500 steps in the same duct flow grows with the
    capillary number (the paper's trend: larger Ca, larger deformation)."""
    geo = G.straight_duct(96, 28, 28, 24.0, u_max=0.03)
    D = []
    for Ca in (0.03, 0.1):
        V, T = Ms.sphere_mesh(642, 12.0, (14.0, geo.info["yc"] + 1.0, geo.info["zc"]), Ms.SplitMix64(5))
        s = gpu_for(case(geo, u_max=0.03, capsules=[W._capsule(V, T, Ca=Ca, u_ref=0.03)]))
        s.step(1500)
        D.append(s.read_capsule(0)["taylor_D"])
    print(f"Taylor D after 1500 steps: Ca 0.03 -> {D[0]:.4e}, Ca 0.1 -> {D[1]:.4e}")
    assert 0.0 < D[0] < D[1], D
