"""The paper's own set-up as inputs (Section "Computational set-up and
boundary conditions"): the circular-duct bifurcation with its sharp and
flat-topped junctions and the capsule meshes with the listed marker counts
(no GPU)."""
import math

import numpy as np
import pytest

from oracle import membrane
from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W


@pytest.fixture(scope="module")
def sharp_and_smooth():
    return G.circular_bifurcation(30.0, 30.0, smooth=False), G.circular_bifurcation(30.0, 30.0, smooth=True)


def test_duct_cross_sections(sharp_and_smooth):
    """Fluid nodes of a main-duct cross-section ~ pi d^2 / 4 (d = 30) and of the
    inlet face the same; the inlet carries a circular Poiseuille profile whose
    peak is u_max on the axis."""
    g, _ = sharp_and_smooth
    t3 = g.tag.reshape(g.nz, g.ny, g.nx)
    n_sec = int((t3[:, :, 100] == 0).sum())
    assert abs(n_sec - math.pi * 15.0 ** 2) < 0.03 * math.pi * 15.0 ** 2
    vel = g.faces[0].velocity
    assert g.faces[0].kind == G.FACE_VELOCITY
    assert np.isclose(vel[:, 0].max(), g.info["u_max"], rtol=1e-2)
    inlet_fluid = (t3[:, :, 0] == 0).reshape(-1)
    assert not (vel[:, 0] > 0)[~inlet_fluid].any()


def test_daughters_and_junction(sharp_and_smooth):
    """Daughters of diameter 0.7 d leave at +-30 deg; the flat-topped junction
    differs from the sharp one only by the filled tip of the cusp between the
    daughters, which ends in a face d / 3 wide at x_cut."""
    sharp, smooth = sharp_and_smooth
    diff = (sharp.tag == 1) & (smooth.tag == 0)
    assert diff.sum() > 0 and not ((sharp.tag == 0) & (smooth.tag == 1)).any()
    n = np.nonzero(diff)[0]
    X, Y = n % sharp.nx, (n // sharp.nx) % sharp.ny
    assert X.min() >= sharp.info["x_cusp"] - 1.5 and X.max() <= smooth.info["x_cut"] + 0.5
    assert np.abs(Y - sharp.info["yc"]).max() <= 30.0 / 6.0 + 1.0
    # a daughter cross-section normal to its axis, away from the junction
    th = math.radians(30.0)
    s = sharp.info["x_junction"] - 15.0
    c = np.array([s, sharp.info["yc"], sharp.info["zc"]]) + 70.0 * np.array([math.cos(th), math.sin(th), 0.0])
    u = np.array([-math.sin(th), math.cos(th), 0.0])
    w = np.array([0.0, 0.0, 1.0])
    a = np.linspace(-14, 14, 57)
    P = c[None, None, :] + a[:, None, None] * u[None, None, :] + a[None, :, None] * w[None, None, :]
    inside = sharp.sdf(P.reshape(-1, 3)) < 0
    area = inside.sum() * (a[1] - a[0]) ** 2
    assert abs(area - math.pi * 10.5 ** 2) < 0.05 * math.pi * 10.5 ** 2


@pytest.mark.parametrize("dp_ratio,n", [(1 / 3, 325), (0.5, 485), (2 / 3, 645), (5 / 6, 785)])
def test_capsule_meshes_with_the_listed_marker_counts(dp_ratio, n):
    """n_L = 325, 485, 645, 785 markers for d_p/d = 1/3 .. 5/6: closed,
    outward meshes (2 n - 4 triangles, every edge in two triangles) whose
    volume is within 2 % of the sphere of diameter d_p."""
    c = W.paper_single_capsule(dp_ratio=dp_ratio)
    cap = c["capsules"][0]
    V, T = cap["verts"], cap["tris"]
    assert V.shape[0] == n and T.shape[0] == 2 * n - 4
    topo = membrane.Topology(T)
    assert topo.edge.shape[0] == 3 * n - 6
    d = membrane.diagnostics(V, T)
    dp = dp_ratio * 30.0
    assert abs(d["volume"] / (math.pi * dp ** 3 / 6) - 1) < 0.02
    assert np.allclose(d["centroid"], [1.16 * 30.0, c["geometry"].info["yc"], c["geometry"].info["zc"]], atol=0.2)


def test_train_of_three_positions():
    c = W.paper_train(kinds=("soft", "rigid", "soft"))
    xs = [membrane.diagnostics(k["verts"], k["tris"])["centroid"][0] for k in c["capsules"]]
    assert np.allclose(np.diff(xs), 0.85 * 30.0, atol=0.3)
    assert [k["params"]["rigid"] for k in c["capsules"]] == [0, 1, 0]
