"""The CUDA discrete adjoint (ibl_adjoint) against the oracle's FP64 adjoint
on the same seeded bifurcation (GPU).  The oracle's adjoint is itself pinned
against central finite differences (tests/test_oracle_adjoint.py); the CUDA
gradients, computed in FP32 with FP64 accumulators, must match it to 1e-3."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import lattice as L
from paper_2207_06043_gb300 import geometry as G

from helpers import case, gpu_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


@pytest.mark.parametrize("steps,ckpt", [(12, 5), (12, 12), (9, 1)])
def test_adjoint_gradients_match_the_oracle(steps, ckpt):
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.02, with_dq=True)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic)
    f = lat.init_equilibrium()
    for _ in range(25):
        f = lat.step(f)
    lo, hi, d = (2, 0, 0), (24, 20, 16), (1.0, 0.3, 0.0)
    J0, gu0, gq0 = A.gradient(lat, f, steps, A.Objective(lo, hi, d), g.links["dq"].astype(np.float64))
    s = gpu_for(case(g))
    s.step(25)
    J1, gu1, gq1 = s.adjoint_flow(steps, lo, hi, d, ckpt_every=ckpt)
    assert J1 == pytest.approx(J0, rel=1e-5)
    assert gu1 == pytest.approx(gu0, rel=1e-3)
    assert gq1 == pytest.approx(gq0, rel=1e-3)
    assert s.member_steps(0) == 25 + steps


def test_adjoint_leaves_the_forward_state_of_plain_steps():
    """The adjoint call advances the context exactly like ibl_step."""
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.02, with_dq=True)
    a = gpu_for(case(g))
    b = gpu_for(case(g))
    a.step(7)
    a.adjoint_flow(11, (2, 0, 0), (24, 20, 16), (1.0, 0.0, 0.0), ckpt_every=4)
    b.step(18)
    assert np.array_equal(a.read_populations(), b.read_populations())


def test_adjoint_rejects_capsules_and_16_bit_storage():
    from paper_2207_06043_gb300 import meshes as Ms
    from paper_2207_06043_gb300 import workloads as W
    from paper_2207_06043_gb300.binding import ERR_STATE, IBLError
    g = G.bifurcation(40, 20, 16, 10.0, 45.0, 3.0, u_max=0.02)
    V, T = Ms.sphere_mesh(162, 6.0, (8.0, g.info["yc"], g.info["zc"]), Ms.SplitMix64(1))
    for s in (gpu_for(case(g, capsules=[W._capsule(V, T, Ca=0.05)])), gpu_for(case(g), "f16")):
        with pytest.raises(IBLError) as e:
            s.adjoint_flow(2, (0, 0, 0), (4, 4, 4), (1.0, 0.0, 0.0))
        assert e.value.status == ERR_STATE
