"""Checkpoint / restart through ibl_save_state / ibl_load_state (GPU): a
context restored from a snapshot continues exactly as the saved one."""
import numpy as np
import pytest

from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms
from paper_2207_06043_gb300 import workloads as W

from helpers import case, gpu_for, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def test_restart_without_capsules_is_bit_identical():
    """No capsules: no atomics, so the continued runs agree bit for bit
    (13 saved steps: the restart begins on an odd AA step)."""
    c = case(G.bifurcation(40, 20, 16, 10.0, 30.0, 2.0))
    a = gpu_for(c)
    a.step(13)
    blob = a.save_state()
    a.step(10)
    b = gpu_for(c)
    b.load_state(blob)
    assert b.member_steps(0) == 13
    b.step(10)
    assert np.array_equal(a.read_populations(), b.read_populations())


def test_restart_with_a_soft_capsule_continues_the_run():
    g = G.bifurcation(48, 20, 20, 14.0, 45.0, 2.0, u_max=0.02)
    V, T = Ms.sphere_mesh(162, 7.0, (10.0, g.info["yc"] + 1.0, g.info["zc"] - 0.5), Ms.SplitMix64(3))
    c = case(g, capsules=[W._capsule(V, T, Ca=0.05)])
    a = gpu_for(c)
    a.step(20)
    blob = a.save_state()
    a.step(15)
    b = gpu_for(c)
    b.load_state(blob)
    b.step(15)
    _, ua = a.read_fields()
    _, ub = b.read_fields()
    # spreading atomics sum in no fixed order: FP32 last-bit differences only
    assert rel_l2(ub, ua, g.tag == 0) <= 1e-6
    xa = a.read_capsule(0, with_verts=True)["verts"]
    xb = b.read_capsule(0, with_verts=True)["verts"]
    assert np.abs(xa - xb).max() <= 1e-6


def test_snapshot_of_another_set_up_is_rejected():
    from paper_2207_06043_gb300.binding import ERR_ARG, IBLError
    a = gpu_for(case(G.periodic_box(12, 10, 8)))
    a.step(2)
    blob = a.save_state()
    b = gpu_for(case(G.periodic_box(12, 10, 9)))
    with pytest.raises(IBLError) as e:
        b.load_state(blob)
    assert e.value.status == ERR_ARG


def test_device_capsule_diagnostics_match_the_host_ones():
    """ibl_read_capsules (FP64 sums on the device, one read for all capsules)
    equals ibl_read_capsule (FP64 sums of the downloaded vertices) for every
    capsule of a context, after some steps, to FP64 rounding (the largest
    stretch to the FP32 rounding of the rest lengths)."""
    from paper_2207_06043_gb300 import meshes as Ms
    from paper_2207_06043_gb300 import workloads as W
    g = G.periodic_box(40, 24, 20)
    caps = []
    for k, ctr in enumerate([(8.0, 10.0, 10.0), (20.0, 12.0, 9.5), (31.0, 11.0, 10.5)]):
        V, T = Ms.sphere_mesh(642 if k == 1 else 162, 8.0, ctr, Ms.SplitMix64(30 + k))
        caps.append(W._capsule(V, T, Ca=0.05, vel0=(0.01, 0.002 * k, 0.0)))
    s = gpu_for(case(g, tau=0.9, capsules=caps))
    s.step(25)
    dev = s.read_capsules(3)
    for k in range(3):
        host = s.read_capsule(k)
        for key in ("centroid", "volume", "area", "dS", "taylor_D", "semi_axes", "velocity"):
            np.testing.assert_allclose(dev[k][key], host[key], rtol=1e-9, atol=1e-12, err_msg=key)
        # the device divides by the FP32 rest lengths that the damage rule uses
        np.testing.assert_allclose(dev[k]["max_stretch"], host["max_stretch"], rtol=1e-7, err_msg="max_stretch")


def test_field_reads_into_pageable_pinned_and_device_buffers_agree():
    """ibl_read_fields into pageable numpy arrays (staged through the
    context's device buffer), into page-locked tensors (written by the read
    kernel directly) and into device tensors: the same values bit for bit."""
    import torch
    c = case(G.bifurcation(40, 20, 16, 10.0, 30.0, 2.0))
    s = gpu_for(c)
    s.step(7)
    r0, u0 = s.read_fields()
    n = r0.shape[0]
    rp = torch.empty(n, dtype=torch.float32, pin_memory=True)
    up = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
    s.read_fields(out=(rp, up))
    rd = torch.empty(n, dtype=torch.float32, device="cuda")
    ud = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    s.read_fields(out=(rd, ud))
    assert np.array_equal(r0, rp.numpy()) and np.array_equal(u0, up.numpy())
    assert np.array_equal(r0, rd.cpu().numpy()) and np.array_equal(u0, ud.cpu().numpy())
    assert np.abs(u0).max() > 0
    with pytest.raises(ValueError):
        s.read_fields(out=(rp, ud))
