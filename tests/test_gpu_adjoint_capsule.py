"""The CUDA discrete adjoint of the coupled step with a soft capsule
(ibl_adjoint) against the oracle's exact derivative of the same discrete run
(the complex step through the whole FP64 oracle, itself pinned against
central differences in tests/test_oracle_adjoint.py), on a seeded bifurcation
with a rounded junction (GPU).  J = D + 0.5 (y_c - y_sym) of the capsule after
the last step; gradients with respect to Ca, u_max and the junction radius."""
import numpy as np
import pytest

from oracle import adjoint as A
from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W

from helpers import case, gpu_for

pytestmark = pytest.mark.gpu

W_D, W_OFF = 1.0, 0.5
GRAD_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _case(dq_scale=0.0, Ca=0.05, u_max=0.03):
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=u_max, with_dq=True)
    if dq_scale:
        g.links["q"] = g.links["q"] + np.float32(dq_scale) * g.links["dq"]
    V, T = Ms.sphere_mesh(162, 7.0, (9.0, g.info["yc"] + 0.4, g.info["zc"] - 0.3), Ms.SplitMix64(4))
    return case(g, u_max=u_max, capsules=[W._capsule(V, T, Ca=Ca, u_ref=0.03)])


@pytest.fixture(scope="module")
def oracle_gradient():
    c = _case()
    return A.coupled_gradient(c, 30, W_D, W_OFF, c["geometry"].info["yc"])


@pytest.mark.parametrize("ckpt", [30, 7])
def test_capsule_adjoint_matches_the_oracle_derivative(oracle_gradient, ckpt):
    """30 coupled steps, one segment (ckpt 30) or five with recompute (ckpt 7):
    the three gradients within 1e-3 relative of the oracle's."""
    J, g_ca, g_um, g_rj = oracle_gradient
    c = _case()
    s = gpu_for(c)
    gc, gu, gr = s.adjoint(30, (W_D, W_OFF), ckpt_every=ckpt)
    st = s.read_capsule(0)
    Jg = W_D * st["taylor_D"] + W_OFF * (st["centroid"][1] - c["geometry"].info["yc"])
    print(f"ckpt {ckpt}: J {Jg:.8e} / {J:.8e}; dJ/dCa {gc:.6e} / {g_ca:.6e}; dJ/du_max {gu:.6e} / {g_um:.6e}; "
          f"dJ/dr_j {gr:.6e} / {g_rj:.6e}")
    assert abs(Jg - J) <= 1e-5 * abs(J)
    for got, ref in ((gc, g_ca), (gu, g_um), (gr, g_rj)):
        assert abs(got - ref) <= GRAD_TOL * abs(ref), (got, ref)


def test_capsule_adjoint_leaves_the_forward_state_of_plain_steps():
    """The adjoint call advances the context like ibl_step (the spreading's
    atomics add in no fixed order, so the two agree to FP32 rounding)."""
    c = _case()
    a = gpu_for(c)
    b = gpu_for(c)
    a.step(4)
    a.adjoint(13, (1.0, 0.0), ckpt_every=5)
    b.step(17)
    assert a.member_steps(0) == b.member_steps(0) == 17
    np.testing.assert_allclose(a.read_populations(), b.read_populations(), atol=1e-6, rtol=0)
    assert np.abs(a.read_capsule(0, with_verts=True)["verts"] - b.read_capsule(0, with_verts=True)["verts"]).max() < 1e-6


def test_capsule_adjoint_rejects_unsupported_contexts():
    from paper_2207_06043_gb300.binding import ERR_STATE, IBLError
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.02)
    V, T = Ms.sphere_mesh(162, 6.0, (8.0, g.info["yc"], g.info["zc"]), Ms.SplitMix64(1))
    bad = [gpu_for(case(g)), gpu_for(case(g, capsules=[W._capsule(V, T, rigid=True)])),
           gpu_for(case(g, capsules=[W._capsule(V, T, Ca=0.05)]), "f16")]
    for s in bad:
        with pytest.raises(IBLError) as e:
            s.adjoint(2, (1.0, 0.0))
        assert e.value.status == ERR_STATE


def test_capsule_objective_autograd_function(oracle_gradient):
    """torch.autograd.Function over (Ca, u_max, r_j): forward gives (D, offset)
    of the capsule, backward the adjoint's gradient of w . (D, offset)."""
    import torch
    from paper_2207_06043_gb300.binding import capsule_objective_function
    J, g_ca, g_um, g_rj = oracle_gradient
    base = _case()

    def build(Ca, u_max, r_j):
        assert r_j == 3.0
        c = _case(Ca=Ca, u_max=u_max)
        return gpu_for(c)

    fn = capsule_objective_function()
    p = torch.tensor([0.05, 0.03, 3.0], dtype=torch.float64, requires_grad=True)
    out = fn.apply(p, build, 30, base["geometry"].info["yc"], 10)
    (W_D * out[0] + W_OFF * out[1]).backward()
    assert abs(float(W_D * out[0] + W_OFF * out[1]) - J) <= 1e-5 * abs(J)
    for got, ref in zip(p.grad.tolist(), (g_ca, g_um, g_rj)):
        assert abs(got - ref) <= GRAD_TOL * abs(ref), (got, ref)
