"""Slab decomposition along x on one GPU (ibl_slab_group_create): the lattice
cut into x-slabs, each a member of one batched context with four ghost planes
per cut side, refreshed from their owners after every step.  Against the
undivided lattice: every population bit for bit after odd and even step
counts, on a bifurcation with an inlet and outlets, a periodic duct, FP16
storage, uneven slabs, and the throughput lattice at full size; with
capsules that cross the cuts (soft and rigid, the throughput workload's 64
included), the fields and the capsules within the rounding of the spreading's
atomics."""
import numpy as np
import pytest

from paper_2207_06043_gb300 import binding as B
from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _pair(g, S, storage="f32", F=(0.0, 0.0, 0.0), u_max=0.03):
    whole = B.Solver.from_geometry(g, 0.8, storage=storage, body_force=F, u_max=u_max)
    grp = B.slab_group(whole, S)
    ref = B.Solver.from_geometry(g, 0.8, storage=storage, body_force=F, u_max=u_max)
    whole.close()
    return grp, ref


def _same_after(grp, ref, steps):
    a, _ = grp.step(steps)
    b, _ = ref.step(steps)
    assert a == b == steps
    ga, gb = grp.read_populations(), ref.read_populations()
    assert np.array_equal(ga.view(np.uint32), gb.view(np.uint32)), float(np.abs(ga - gb).max())
    ra, ua = grp.read_fields()
    rb, ub = ref.read_fields()
    assert np.array_equal(ua, ub) and np.array_equal(ra, rb)
    return float(np.abs(ub).max())


@pytest.mark.parametrize("S", [2, 3])
def test_bifurcation_slabs_bit_for_bit(S):
    g = G.bifurcation(64, 28, 24, 12.0, 45.0, 3.0, u_max=0.03)
    grp, ref = _pair(g, S)
    assert len(grp.slabs) == S
    umax = _same_after(grp, ref, 31)
    assert umax > 1e-3
    _same_after(grp, ref, 16)          # 47 steps in all: the other parity
    grp.close()
    ref.close()


def test_periodic_duct_slabs_bit_for_bit():
    g = G.straight_duct(60, 16, 16, 12.0, periodic_x=True)
    grp, ref = _pair(g, 3, F=(2e-5, 0.0, 0.0))
    assert all(lo == hi == 4 for _, _, lo, hi in grp.slabs)
    assert _same_after(grp, ref, 40) > 1e-4
    grp.close()
    ref.close()


def test_fp16_storage_slabs_bit_for_bit():
    g = G.bifurcation(64, 28, 24, 12.0, 45.0, 3.0, u_max=0.03)
    grp, ref = _pair(g, 2, storage="f16")
    _same_after(grp, ref, 25)
    grp.close()
    ref.close()


def test_throughput_lattice_in_four_slabs():
    """512x192x128 (3.8 M fluid nodes), four slabs balanced by fluid nodes."""
    c = W.throughput_case()
    g = c["geometry"]
    grp, ref = _pair(g, 4, u_max=c["u_max"])
    widths = [x1 - x0 for x0, x1, _, _ in grp.slabs]
    assert sum(widths) == g.nx and len(set(widths)) > 1     # balanced by fluid, not by planes
    assert _same_after(grp, ref, 21) > 1e-3
    grp.close()
    ref.close()


def test_slab_group_rejects_short_halos():
    g = G.bifurcation(48, 20, 16, 10.0, 45.0, 3.0, u_max=0.02)
    whole = B.Solver.from_geometry(g, 0.8, u_max=0.02)
    with pytest.raises(B.IBLError) as e:
        B.slab_group(whole, 2, halo=3)
    assert e.value.status == B.ERR_ARG
    whole.close()


def _with_capsules(c, storage="f32"):
    from helpers import gpu_for
    return gpu_for(c, storage)


def _compare_capsules(c, S, steps):
    from helpers import rel_l2
    whole = _with_capsules(c)
    grp = B.slab_group(whole, S)
    ref = _with_capsules(c)
    whole.close()
    a, _ = grp.step(steps)
    b, _ = ref.step(steps)
    assert a == b == steps
    _, ua = grp.read_fields()
    _, ub = ref.read_fields()
    fluid = c["geometry"].tag == 0
    err = rel_l2(ua, ub, fluid)
    n = len(c["capsules"])
    dc = max(float(np.abs(grp.read_capsule(k)["centroid"] - ref.read_capsule(k)["centroid"]).max())
             for k in range(n))
    sa, sb = grp.read_capsules(n), ref.read_capsules(n)
    dD = max(abs(x["taylor_D"] - y["taylor_D"]) for x, y in zip(sa, sb))
    grp.close()
    ref.close()
    return err, dc, dD


def test_capsules_across_the_cuts():
    """A bifurcation (96x40x32) with three soft capsules and a rigid sphere
    placed across the cuts of two and three slabs: after 200 steps the
    velocity relative L2 <= 1e-5 and every centroid within 1e-4 lu of the
    undivided lattice's."""
    from paper_2207_06043_gb300 import workloads as W
    g = G.bifurcation(96, 40, 32, 20.0, 45.0, 3.0, u_max=0.03)
    yc, zc = g.info["yc"], g.info["zc"]
    caps = []
    for k, (x, rigid) in enumerate(((30.0, False), (47.0, False), (64.0, True), (20.0, False))):
        V, T = Ms.sphere_mesh(642, 9.0, (x, yc + (k % 2) * 1.5 - 0.7, zc + 0.4), Ms.SplitMix64(40 + k))
        caps.append(W._capsule(V, T, rigid=rigid, Ca=0.05, u_ref=0.03))
    from helpers import case
    c = case(g, u_max=0.03, capsules=caps)
    for S in (2, 3):
        err, dc, dD = _compare_capsules(c, S, 200)
        print(f"{S} slabs, 4 bodies, 200 steps: u rel L2 {err:.2e}, centroid {dc:.2e}, Taylor D {dD:.2e}")
        assert err <= 1e-5 and dc <= 1e-4 and dD <= 1e-5, (S, err, dc, dD)


def test_throughput_workload_in_four_slabs():
    """The throughput workload (512x192x128, 64 capsules) in four slabs:
    50 steps against the undivided context, velocity rel L2 <= 1e-5 and
    centroids within 1e-4 lu."""
    c = W.throughput_case()
    err, dc, dD = _compare_capsules(c, 4, 50)
    print(f"throughput workload, 4 slabs, 50 steps: u rel L2 {err:.2e}, centroid {dc:.2e}, Taylor D {dD:.2e}")
    assert err <= 1e-5 and dc <= 1e-4, (err, dc)
