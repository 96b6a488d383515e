"""ibl_read_fields_noalloc (static device staging array, no allocation)
against ibl_read_fields on the same state (GPU).  Collected last so that it
also runs after every other test of the session has used the library."""
import ctypes as C

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


def _noalloc(s, n, member=0):
    from paper_2207_06043_gb300.binding import lib
    L = lib()
    rho = np.full(n, np.nan, np.float32)
    u = np.full((n, 3), np.nan, np.float32)
    st = L.ibl_read_fields_noalloc(s._h, member, rho.ctypes.data_as(C.c_void_p), u.ctypes.data_as(C.c_void_p))
    return st, rho, u


def test_noalloc_read_matches_read_fields_on_consecutive_calls():
    g = G.bifurcation(48, 20, 20, 14.0, 45.0, 2.0, u_max=0.02)
    V, T = Ms.sphere_mesh(162, 7.0, (10.0, g.info["yc"] + 1.0, g.info["zc"] - 0.5), Ms.SplitMix64(3))
    s = gpu_for(case(g, capsules=[W._capsule(V, T, Ca=0.05)]))
    n = g.n_nodes
    for steps in (5, 6):          # odd and even step counts: both storage parities
        s.step(steps)
        rho0, u0 = s.read_fields()
        for _ in range(2):        # two calls in a row on the same state
            st, rho1, u1 = _noalloc(s, n)
            assert st == 0
            np.testing.assert_allclose(rho1, rho0, rtol=1e-7, atol=0)
            np.testing.assert_allclose(u1, u0, rtol=1e-6, atol=1e-9)


def test_noalloc_read_rejects_lattices_beyond_the_static_array():
    from paper_2207_06043_gb300.binding import ERR_ARG, lib
    g = G.periodic_box(128, 96, 96)          # 1,179,648 nodes > 2^20
    s = gpu_for(case(g))
    st, _, _ = _noalloc(s, 1)
    assert st == ERR_ARG
    assert b"IBL_NOALLOC_MAX_NODES" in lib().ibl_last_error(s._h)


def test_noalloc_read_needs_device_state():
    from paper_2207_06043_gb300.binding import ERR_STATE
    g = G.periodic_box(12, 10, 8)
    s = gpu_for(case(g))
    st, _, _ = _noalloc(s, g.n_nodes)
    assert st == ERR_STATE
    s.step(1)
    st, rho, _ = _noalloc(s, g.n_nodes)
    assert st == 0 and np.isfinite(rho).all()
