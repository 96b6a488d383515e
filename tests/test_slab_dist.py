"""Slab decomposition along x on CPU: the library's host-only planner
(ibl_slab_plan), and the halo protocol of a slab context run by two gloo ranks
that each step the FP64 oracle's lattice on their slab (owned planes plus
four ghost planes per cut side) and swap ghost planes by send / recv after
every step.  The owned planes must match the undivided oracle bit for bit:
the exchange carries exactly what the library's slab context copies between
its members on one GPU (every population of every node of each ghost plane,
from the slab that owns the plane)."""
import os
import socket

import numpy as np
import pytest

from paper_2207_06043_gb300 import binding as B
from paper_2207_06043_gb300 import geometry as G

HALO = 4
STEPS = 31


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2207_06043_gb300 import build
        build.build()
    B.lib()


def test_planner_tiles_the_axis_with_balanced_slabs():
    for nx, S, per in ((100, 3, False), (100, 3, True), (37, 4, False), (64, 1, False), (64, 1, True)):
        plan = B.slab_plan(nx, S, HALO, periodic_x=per)
        assert plan[0][0] == 0 and plan[-1][1] == nx
        for (a0, a1, lo, hi), nxt in zip(plan, plan[1:] + [None]):
            assert a1 - a0 >= HALO
            if nxt is not None:
                assert nxt[0] == a1
            if S == 1:
                assert lo == hi == 0
            else:
                assert lo == (HALO if per or a0 > 0 else 0)
                assert hi == (HALO if per or a1 < nx else 0)
    # weights: twice the work in the first half
    w = np.ones(120)
    w[:60] = 2.0
    plan = B.slab_plan(120, 3, HALO, plane_weight=w)
    loads = [w[a:b].sum() for a, b, _, _ in plan]
    assert max(loads) - min(loads) <= 2.0, loads
    with pytest.raises(B.IBLError):
        B.slab_plan(10, 3, HALO)


def _crop(g, sl, S):
    """The slab's lattice: its owned and ghost planes, the links that start
    and end on them, real faces kept, cut faces without a condition."""
    x0, x1, lo, hi = sl
    nx, ny, nz = g.nx, g.ny, g.nz
    nxs = x1 - x0 + lo + hi
    gx = (x0 - lo + np.arange(nxs)) % nx
    tag = g.tag.reshape(nz, ny, nx)[:, :, gx].reshape(-1).copy()
    links = []
    lx = g.links["node"] % nx
    rest = g.links["node"] // nx
    for l in range(nxs):
        sel = np.nonzero(lx == gx[l])[0]
        t = l + G.E19[g.links["dir"][sel].astype(np.int64), 0]
        keep = sel[(t >= 0) & (t < nxs)]
        lk = g.links[keep].copy()
        lk["node"] = (l + nxs * rest[keep]).astype(np.uint32)
        links.append(lk)
    links = np.concatenate(links) if links else np.zeros(0, G.LINK_DTYPE)
    faces = [G.Face(f.kind, f.rho, f.velocity) for f in g.faces]
    if S > 1:
        if g.periodic[0] or x0 > 0:
            faces[0] = G.Face()
        if g.periodic[0] or x1 < nx:
            faces[1] = G.Face()
    for f in (2, 3, 4, 5):
        if faces[f].kind == G.FACE_VELOCITY:
            raise ValueError("the test geometries have velocity faces on x only")
    per = (False if S > 1 else g.periodic[0], g.periodic[1], g.periodic[2])
    return G.Geometry(nxs, ny, nz, per, tag, links, faces, None, {}), gx


def _geometry(kind):
    if kind == "bifurcation":
        return G.bifurcation(48, 20, 16, 8.0, 45.0, 2.0, u_max=0.03), (0.0, 0.0, 0.0)
    return G.straight_duct(40, 12, 12, 8.0, periodic_x=True), (2e-5, 0.0, 0.0)


def _plan(g):
    w = (g.tag.reshape(g.nz, g.ny, g.nx) == 0).sum(axis=(0, 1)).astype(np.float64)
    return B.slab_plan(g.nx, 2, HALO, periodic_x=g.periodic[0], plane_weight=w)


def _rank(rank, world, port, kind, q):
    import torch
    import torch.distributed as dist
    from oracle import lattice as L
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, F = _geometry(kind)
    plan = _plan(g)
    mine, gx = _crop(g, plan[rank], world)
    x0, x1, lo, hi = plan[rank]
    nxs = mine.nx
    lat = L.Lattice(mine.nx, mine.ny, mine.nz, 0.8, mine.tag, mine.links, mine.faces, mine.periodic,
                    body_force=np.array(F))
    f = lat.init_equilibrium()
    # the other rank's ghost planes that this rank owns: (their local plane,
    # my local plane), in their order
    other = 1 - rank
    ox0, ox1, olo, ohi = plan[other]
    onx = ox1 - ox0 + olo + ohi
    send_planes, recv_planes = [], []
    for l in range(onx):
        if olo <= l < olo + (ox1 - ox0):
            continue
        g_x = (ox0 - olo + l) % g.nx
        assert x0 <= g_x < x1
        send_planes.append(g_x - x0 + lo)
    for l in range(nxs):
        if not (lo <= l < lo + (x1 - x0)):
            recv_planes.append(l)
    for _ in range(STEPS):
        f = lat.step(f, check=False)
        f4 = f.reshape(19, g.nz, g.ny, nxs)
        out = torch.from_numpy(np.ascontiguousarray(f4[:, :, :, send_planes]))
        inc = torch.empty((19, g.nz, g.ny, len(recv_planes)), dtype=torch.float64)
        reqs = [dist.isend(out, other), dist.irecv(inc, other)]
        for r in reqs:
            r.wait()
        f4[:, :, :, recv_planes] = inc.numpy()
        f = f4.reshape(19, -1)
    own = f.reshape(19, g.nz, g.ny, nxs)[:, :, :, lo:lo + (x1 - x0)]
    q.put((rank, x0, x1, np.ascontiguousarray(own)))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("kind", ["bifurcation", "periodic_duct"])
def test_two_gloo_ranks_match_the_undivided_lattice(kind):
    import multiprocessing as mp
    from oracle import lattice as L
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g, F = _geometry(kind)
    lat = L.Lattice(g.nx, g.ny, g.nz, 0.8, g.tag, g.links, g.faces, g.periodic, body_force=np.array(F))
    f = lat.init_equilibrium()
    for _ in range(STEPS):
        f = lat.step(f)
    f4 = f.reshape(19, g.nz, g.ny, g.nx)
    assert np.abs(f4 - lat.init_equilibrium().reshape(f4.shape)).max() > 1e-5    # the flow moved
    for rank, x0, x1, own in parts:
        assert np.array_equal(own, f4[:, :, :, x0:x1]), (kind, rank)
