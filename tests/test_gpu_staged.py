"""The staged lattice kernel (every run of consecutive interior fluid nodes cut
into chunks whose populations and tags are fetched into shared memory by bulk
copies) against the register-gather kernel and the FP64 oracle (GPU).

Long ducts along x give long runs (the work list runs along x rows), and a
length that is not a multiple of the chunk leaves short chunks and idle lanes
at every row end.  Tolerances as in test_gpu_parity.py."""
import numpy as np
import pytest

from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W

from helpers import case, gpu_for, oracle_for, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _duct(nx=150, n=24, D=20.0, u=0.03):
    return G.straight_duct(nx, n, n, D, u_max=u)


def test_staged_path_is_opt_in_and_for_one_lattice_only():
    g = _duct(96, 16, 12.0)
    s = gpu_for(case(g, u_max=0.03))
    assert s.lattice_path() == -1
    s.step(1)
    assert s.lattice_path() == 0
    s.set_lattice_path(True)
    assert s.lattice_path() == 1
    s.step(1)
    s.set_lattice_path(False)
    assert s.lattice_path() == 0
    from paper_2207_06043_gb300.binding import ensemble
    a = gpu_for(case(g, u_max=0.03))
    b = gpu_for(case(g, u_max=0.03))
    a.set_lattice_path(True)
    ens = ensemble([a, b])
    ens.set_lattice_path(True)
    ens.step(1)
    assert ens.lattice_path() == 0
    for x in (ens, a, b, s):
        x.close()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("steps", [30, 31])
def test_staged_equals_register_kernel_without_capsules(storage, steps):
    """Same populations, bit for bit, after an even and an odd number of
    steps (both AA parities end a run): the two kernels load the same slots
    and share the collision code."""
    g = _duct()
    c = case(g, u_max=0.03)
    a = gpu_for(c, storage=storage)
    b = gpu_for(c, storage=storage)
    a.set_lattice_path(True)
    a.step(steps)
    b.step(steps)
    assert a.lattice_path() == 1 and b.lattice_path() == 0
    ga, gb = a.read_populations(), b.read_populations()
    assert np.array_equal(ga, gb), float(np.abs(ga - gb).max())
    a.close()
    b.close()


def test_staged_against_oracle_soft_capsule_in_long_duct():
    g = _duct(118, 24, 20.0)
    V, T = Ms.sphere_mesh(642, 12.0, (14.0, g.info["yc"] + 0.7, g.info["zc"] - 0.4), Ms.SplitMix64(11))
    c = case(g, u_max=0.03, capsules=[W._capsule(V, T, Ca=0.05, Eb=0.01, u_ref=0.03)])
    lat, o = oracle_for(c)
    s = gpu_for(c)
    s.set_lattice_path(True)
    steps = 80
    s.step(steps)
    assert s.lattice_path() == 1
    o.step(steps)
    _, u = s.read_fields()
    _, uo = lat.macroscopic(o.f)
    err = rel_l2(u, uo, lat.fluid)
    dc = np.abs(s.read_capsule(0)["centroid"] - o.stats(0)["centroid"]).max()
    assert err <= 1e-5 and dc <= 1e-4, (err, dc)
    s.close()


def test_staged_and_register_kernels_agree_with_capsules():
    """With capsules the spread IB force is summed by atomics (order not
    fixed), so the two runs agree to rounding, not bit for bit."""
    g = _duct(150, 28, 24.0)
    V, T = Ms.sphere_mesh(642, 14.0, (16.0, g.info["yc"], g.info["zc"] + 0.5), Ms.SplitMix64(3))
    c = case(g, u_max=0.03, capsules=[W._capsule(V, T, Ca=0.05, Eb=0.01, u_ref=0.03)])
    a = gpu_for(c)
    b = gpu_for(c)
    a.set_lattice_path(True)
    a.step(61)
    b.step(61)
    _, ua = a.read_fields()
    _, ub = b.read_fields()
    assert rel_l2(ua, ub) <= 1e-6
    dc = np.abs(a.read_capsule(0)["centroid"] - b.read_capsule(0)["centroid"]).max()
    assert dc <= 1e-5, dc
    a.close()
    b.close()
