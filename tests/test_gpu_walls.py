"""Marker-based wall tagging on the GPU (ibl_voxelise_markers; Section
"Boundary conditions on fixed bodies", Eq. qbouzidi) against the oracle
(oracle/walls.py): the tags, the links and every q bit for bit, on a periodic
tube, a fixed sphere in a box with pre-tagged edges, random triangle soups
over periodic axes, a mesh partly outside the box, an empty mesh, and a
256x96x64 box holding a tube of about 10^6 triangles.  Then the coupled step
on a tube given only by its triangulation, against the oracle's lattice on
the same tags and links."""
import numpy as np
import pytest

from oracle import lattice as L
from oracle import walls as Wl
from paper_2207_06043_gb300 import binding as B
from paper_2207_06043_gb300 import geometry as G
from paper_2207_06043_gb300 import meshes as Ms

from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _edges(shape):
    nx, ny, nz = shape
    n = np.arange(nx * ny * nz)
    X, Y, Z = n % nx, (n // nx) % ny, n // (nx * ny)
    on = ((X == 0) | (X == nx - 1)).astype(int) + ((Y == 0) | (Y == ny - 1)) + ((Z == 0) | (Z == nz - 1))
    return (on >= 2).astype(np.uint8)


def _same(V, T, shape, periodic=(False, False, False), tag_in=None):
    tag_o, node_o, dir_o, q_o = Wl.voxelise_markers(V, T, shape, periodic, tag_in)
    tag_g, links = B.voxelise_markers(V, T, shape, periodic, tag_in)
    assert np.array_equal(tag_g, tag_o)
    assert np.array_equal(links["node"], node_o)
    assert np.array_equal(links["dir"], dir_o)
    assert np.array_equal(links["q"].view(np.uint32), q_o.view(np.uint32))
    return len(node_o)


def _tube(R, nx, h=0.3):
    n = int(2 * R + 6)
    c = (n - 1) / 2.0
    V, T = Ms.tube_mesh(-0.5, nx - 0.5, R, c, c, h, periodic_x=True)
    idx = np.arange(nx * n * n)
    r = np.hypot((idx // nx) % n - c, idx // (nx * n) - c)
    return V, T, (nx, n, n), (r > R + 1.5).astype(np.uint8), r


def test_voxelisation_matches_the_oracle_bit_for_bit():
    V, T, shape, tag_in, _ = _tube(6.0, 8)
    counts = [_same(V, T, shape, (True, False, False), tag_in)]
    Vs, Ts = Ms.sphere_mesh(10242, 10.0, (11.3, 9.7, 10.2), Ms.SplitMix64(3))
    counts.append(_same(Vs, Ts, (24, 20, 20), tag_in=_edges((24, 20, 20))))
    rng = np.random.default_rng(11)
    for shape, periodic in (((9, 8, 7), (True, False, True)), ((8, 8, 8), (True, True, True)),
                            ((10, 7, 6), (False, False, False))):
        Vr = rng.uniform(-1.5, max(shape) + 1.0, size=(60, 3))
        Tr = rng.integers(0, 60, size=(120, 3))
        t_in = (rng.uniform(size=int(np.prod(shape))) < 0.04).astype(np.uint8)
        counts.append(_same(Vr, Tr, shape, periodic, t_in))
    # a sphere half outside a non-periodic box: its markers there are dropped
    Vh, Th = Ms.sphere_mesh(2562, 12.0, (1.0, 8.0, 8.0), Ms.SplitMix64(5))
    counts.append(_same(Vh, Th, (16, 16, 16)))
    # no triangles: every link toward a pre-tagged node takes q = 1/2
    n_empty = _same(np.zeros((0, 3)), np.zeros((0, 3), np.int32), (6, 5, 4), tag_in=_edges((6, 5, 4)))
    counts.append(n_empty)
    assert min(counts[:-1]) > 0 and n_empty > 0, counts


def test_voxelisation_at_size():
    """256x96x64 box (1.57 M nodes), tube R = 30 along x, ~1.1 M triangles."""
    R, nx = 30.0, 256
    n0, n1 = 96, 64
    c1, c2 = (n0 - 1) / 2.0, (n1 - 1) / 2.0 + 0.3
    R2 = min(R, (n1 - 6) / 2.0)
    V, T = Ms.tube_mesh(-0.5, nx - 0.5, R2, c1, c2, 0.35, periodic_x=True)
    assert T.shape[0] > 5e5
    nl = _same(V, T, (nx, n0, n1), (True, False, False))
    assert nl > 1e5


def test_voxelisation_errors():
    V = np.zeros((3, 3))
    with pytest.raises(B.IBLError) as e:
        B.voxelise_markers(V, [[0, 1, 3]], (4, 4, 4))
    assert e.value.status == B.ERR_ARG
    # buffers smaller than the link count: IBL_ERR_ARG and the count returned
    import ctypes as C
    Lb = B.lib()
    Vs, Ts = Ms.sphere_mesh(642, 6.0, (6.0, 6.0, 6.0), Ms.SplitMix64(1))
    Vs = np.ascontiguousarray(Vs)
    Ts = np.ascontiguousarray(Ts, dtype=np.int32)
    tag = np.empty(12 ** 3, np.uint8)
    node = np.empty(4, np.uint32)
    dirs = np.empty(4, np.uint32)
    q = np.empty(4, np.float32)
    n = C.c_int64(4)
    per = np.zeros(3, np.int32)
    st = Lb.ibl_voxelise_markers(B._ptr(Vs), Vs.shape[0], B._ptr(Ts), Ts.shape[0], 12, 12, 12, B._ptr(per), None,
                                 B._ptr(tag), B._ptr(node), B._ptr(dirs), B._ptr(q), C.byref(n), None)
    assert st == B.ERR_ARG and n.value > 4


def test_tube_flow_on_marker_walls_matches_the_oracle():
    """Body-force flow through a periodic tube (R = 6) tagged by its markers:
    300 coupled steps of the CUDA path against the oracle's lattice on the
    same tags and links (velocity relative L2 <= 1e-5)."""
    V, T, shape, tag_in, r = _tube(6.0, 8)
    tag, links = B.voxelise_markers(V, T, shape, (True, False, False), tag_in)
    nx, ny, nz = shape
    faces = [G.Face() for _ in range(6)]
    geom = G.Geometry(nx, ny, nz, (True, False, False), tag, links, faces, None, dict(kind="marker_tube"))
    tau, F = 0.8, (2e-5, 0.0, 0.0)
    s = B.Solver.from_geometry(geom, tau, body_force=F, u_max=0.02)
    done, _ = s.step(300)
    assert done == 300
    _, u = s.read_fields()
    s.close()
    lat = L.Lattice(nx, ny, nz, tau, tag, links, faces, (True, False, False), body_force=np.array(F))
    f = lat.init_equilibrium()
    for _ in range(300):
        f = lat.step(f)
    _, uo = lat.macroscopic(f)
    err = rel_l2(u, uo, lat.fluid)
    print(f"marker tube, 300 steps: u rel L2 {err:.2e}, peak {uo[:, 0].max():.4e}")
    assert uo[:, 0].max() > 1e-3
    assert err <= 1e-5, err
