"""CUDA path against the FP64 oracle on the standard workloads (GPU):
the small bifurcation with a rigid sphere over its full 500 steps, the damage
rule, and a per-node check at the throughput workload's full size in the
launch configuration bench.py times."""
import numpy as np
import pytest

from oracle import lattice as L
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


def test_small_bifurcation_rigid_sphere_500_steps():
    """96x32x32 Y-bifurcation, rigid sphere d = 12 (642 v), 500 steps:
    velocity relative L2 <= 1e-5 and centroid within 1e-4 lu of the oracle."""
    c = W.bifurcation_small()
    lat, o = oracle_for(c)
    s = gpu_for(c)
    done, _ = s.step(c["steps"])
    assert done == c["steps"]
    o.step(c["steps"])
    _, u = s.read_fields()
    _, uo = lat.macroscopic(o.f)
    err = rel_l2(u, uo, lat.fluid)
    dc = np.abs(s.read_capsule(0)["centroid"] - o.stats(0)["centroid"]).max()
    assert err <= 1e-5, err
    assert dc <= 1e-4, dc


def test_damage_rule_stops_at_the_oracle_step():
    """A stiff, light capsule (Ca = 0.005, d = 10, 642 v) exceeds the explicit
    stability limit and an edge doubles within a few tens of steps.  The step
    at which the growing mode crosses the threshold depends on its seed, which
    FP32 and FP64 round differently, so the two paths must stop within 25 % of
    each other; the GPU must report the damage and stop stepping."""
    from paper_2207_06043_gb300.binding import ERR_DAMAGED
    g = G.bifurcation(64, 28, 24, 16.0, 45.0, 2.0, u_max=0.02)
    V, T = Ms.sphere_mesh(642, 10.0, (12.0, g.info["yc"], g.info["zc"] + 0.5), Ms.SplitMix64(9))
    c = case(g, capsules=[W._capsule(V, T, Ca=0.005)])
    lat, o = oracle_for(c)
    n_o = o.step(200)
    assert o.damaged
    s = gpu_for(c)
    done, st = s.step(200, allow_damage=True)
    assert st == ERR_DAMAGED
    assert abs(done - n_o) <= max(1, 0.25 * n_o), (done, n_o)
    assert s.read_capsule(0)["damaged"]
    # a damaged lattice stops stepping
    done2, st2 = s.step(5, allow_damage=True)
    assert done2 == 0 and st2 == ERR_DAMAGED


def _sample_nodes(geom, caps, rng, n_interior=3000, n_wall=1500, clear=4.5):
    """Fluid nodes off the box faces and farther than `clear` from every marker
    (no IB force there); some with wall links, the rest interior."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    n = np.arange(geom.n_nodes)
    X, Y, Z = n % nx, (n // nx) % ny, n // (nx * ny)
    ok = (geom.tag == 0) & (X > 0) & (X < nx - 1) & (Y > 0) & (Y < ny - 1) & (Z > 0) & (Z < nz - 1)
    marker = np.zeros(geom.n_nodes, bool)
    for c in caps:
        lo = np.floor(c["verts"].min(0) - clear).astype(int)
        hi = np.ceil(c["verts"].max(0) + clear).astype(int)
        box = (X >= lo[0]) & (X <= hi[0]) & (Y >= lo[1]) & (Y <= hi[1]) & (Z >= lo[2]) & (Z <= hi[2])
        marker |= box
    ok &= ~marker
    wall_nodes = np.unique(geom.links["node"])
    wall = np.zeros(geom.n_nodes, bool)
    wall[wall_nodes] = True
    a = rng.choice(np.nonzero(ok & ~wall)[0], n_interior, replace=False)
    b = rng.choice(np.nonzero(ok & wall)[0], n_wall, replace=False)
    return np.concatenate([a, b])


def test_throughput_workload_full_size_sampled_step():
    """512x192x128, 64 capsules, in the bench launch shape: after a few steps,
    every population of sampled nodes after one more step equals the oracle's
    collision of the upstream nodes (plus the wall rule on wall links),
    computed one node at a time from the GPU's own pre-step populations."""
    c = W.throughput_case()
    g = c["geometry"]
    s = W.make_solver(c)
    s.set_launch(128, 0)
    s.step(3)
    g0 = s.read_populations().astype(np.float64)
    s.step(1)
    g1 = s.read_populations().astype(np.float64)
    rng = np.random.default_rng(1)
    nodes = _sample_nodes(g, c["capsules"], rng)
    nx, ny, nz = g.nx, g.ny, g.nz
    tag = g.tag
    fluid = tag == 0
    W19 = L.W[:, None]

    def idx(x, y, z):
        return x + nx * (y + ny * z)

    def fstar(ids):
        """Oracle collision of the pre-step populations at nodes ids."""
        f = g0[:, ids] + W19
        return L.collide(f, np.zeros((len(ids), 3)), c["tau"])

    X, Y, Z = nodes % nx, (nodes // nx) % ny, nodes // (nx * ny)
    links = {}
    for (node, d, q) in zip(g.links["node"], g.links["dir"], g.links["q"]):
        links[(int(node), int(d))] = float(q)
    worst = 0.0
    for i in range(19):
        e = L.E[i]
        src = idx(X - e[0], Y - e[1], Z - e[2])
        from_fluid = fluid[src]
        # streamed populations
        ids = nodes[from_fluid]
        if ids.size:
            exp = fstar(src[from_fluid])[i] - L.W[i]
            worst = max(worst, float(np.abs(g1[i, ids] - exp).max()))
        # populations returned by a wall link in direction opp(i)
        ib = L.OPP[i]
        for nd in nodes[~from_fluid]:
            q = links[(int(nd), int(ib))]
            x, y, z = nd % nx, (nd // nx) % ny, nd // (nx * ny)
            eb = L.E[ib]
            m1 = idx(x - eb[0], y - eb[1], z - eb[2])
            m2 = idx(x - 2 * eb[0], y - 2 * eb[1], z - 2 * eb[2])
            ok1, ok2 = bool(fluid[m1]), bool(fluid[m2])
            fb = fstar(np.array([nd]))[:, 0]
            f1 = fstar(np.array([m1]))[:, 0] if ok1 else np.zeros(19)
            f2 = fstar(np.array([m2]))[:, 0] if ok2 else np.zeros(19)
            val = L.bouzidi_value(q, fb[ib], f1[ib], f2[ib], fb[i], f1[i], ok1, ok2)
            worst = max(worst, abs(g1[i, nd] - (float(val) - L.W[i])))
    assert worst <= 2e-7, worst


def _face_slab_check(geom, face, tau, g1):
    """The Zou-He rule of one box face on the GPU's own populations: the
    3-node slab along the face becomes an oracle lattice holding only that
    face's condition; the populations entering from outside are blanked and
    refilled by the oracle's rule from the known ones (streamed and wall
    values as the GPU left them).  Returns (face nodes, largest difference)."""
    nx, ny, nz = geom.nx, geom.ny, geom.nz
    ax, side = face // 2, face % 2
    dims = [nx, ny, nz]
    sub = list(dims)
    sub[ax] = 3
    lo = 0 if side == 0 else dims[ax] - 3
    zz, yy, xx = np.meshgrid(np.arange(sub[2]), np.arange(sub[1]), np.arange(sub[0]), indexing="ij")
    cc = [xx.reshape(-1), yy.reshape(-1), zz.reshape(-1)]
    cc[ax] = cc[ax] + lo
    full = cc[0] + nx * (cc[1] + ny * cc[2])
    faces = [None] * 6
    faces[face] = geom.faces[face]
    lat = L.Lattice(sub[0], sub[1], sub[2], tau, geom.tag[full], dict(node=[], dir=[], q=[]), faces, geom.periodic)
    nodes, _ = lat.face_nodes(face)
    f = g1[:, full].astype(np.float64) + L.W[:, None]
    unk = np.nonzero(L.E @ L.FACE_NORMALS[face] < 0)[0]
    for k in unk:
        f[k, nodes] = np.nan
    lat.zou_he(f)
    exp = f[np.ix_(unk, nodes)] - L.W[unk][:, None]
    got = g1[np.ix_(unk, full[nodes])].astype(np.float64)
    return nodes.size, float(np.abs(exp - got).max()) if nodes.size else 0.0


def test_throughput_workload_full_size_ib_structure_and_faces():
    """512x192x128, 64 capsules (163,968 markers), in the bench launch shape:
    one GPU step from its own state after three steps against the oracle's
    operators applied to that same state (populations, x(t), x(t - dt), vertex
    velocities):
      - every vertex's x(t + dt) and velocity: the oracle's marker stencils
        (u_v,0 = U_l), probe stresses, membrane, volume and repulsion forces
        and Verlet update (Eqs. uLag .. verletPosC), within 1e-6 lu;
      - the populations streamed into sampled IB-shell nodes: the oracle's
        spreading (Eq. bodyforce) of every marker's force and the collision
        with it, within 2e-7;
      - every population the Zou-He rule writes at every node of every
        inlet and outlet face, within 2e-7."""
    from types import SimpleNamespace
    from oracle import sim
    c = W.throughput_case()
    g = c["geometry"]
    s = W.make_solver(c)
    s.set_launch(128, 0)
    s.step(3)
    nvs = [len(cap["verts"]) for cap in c["capsules"]]
    g0 = s.read_populations()
    st0 = [s.read_capsule_state(k, nv) for k, nv in enumerate(nvs)]
    s.step(1)
    g1 = s.read_populations()
    st1 = [s.read_capsule_state(k, nv) for k, nv in enumerate(nvs)]
    s.close()
    # the oracle's coupled operators on the GPU's pre-step state
    lat = SimpleNamespace(nx=g.nx, ny=g.ny, nz=g.nz, N=g.n_nodes, tau=c["tau"], periodic=g.periodic,
                          fluid=g.tag == 0)
    o = sim.Simulation.__new__(sim.Simulation)
    o.lat, o.u_max, o.t, o.damaged, o.last = lat, c["u_max"], 0, False, {}
    o.f = g0.astype(np.float64) + L.W[:, None]
    o.bodies = []
    for cap, st in zip(c["capsules"], st0):
        b = sim.Body(cap["verts"], cap["tris"], cap["params"], c["tau"], cap.get("vel0"))
        b.x, b.x_prev, b.vel = st["x"].copy(), st["x_prev"].copy(), st["vel"].copy()
        o.bodies.append(b)
    f_ib, per = o.ib_force()
    o.update(o.f, per, o.structure(o.f, per))
    dx = max(float(np.abs(b.x - st["x"]).max()) for b, st in zip(o.bodies, st1))
    dv = max(float(np.abs(b.vel - st["vel"]).max()) for b, st in zip(o.bodies, st1))
    # streamed populations of sampled shell nodes whose 19 upstream nodes are fluid
    nx, ny, nz = g.nx, g.ny, g.nz
    n = np.arange(g.n_nodes)
    X, Y, Z = n % nx, (n // nx) % ny, n // (nx * ny)
    shell = np.nonzero((np.abs(f_ib).sum(axis=1) > 0) & (X > 1) & (X < nx - 2) & (Y > 1) & (Y < ny - 2)
                       & (Z > 1) & (Z < nz - 2))[0]
    fluid = g.tag == 0
    srcs = [shell - (L.E[i, 0] + nx * (L.E[i, 1] + ny * L.E[i, 2])) for i in range(19)]
    allf = np.all([fluid[sr] for sr in srcs], axis=0)
    rng = np.random.default_rng(3)
    pick = rng.choice(shell[allf], 4000, replace=False)
    worst_ib = 0.0
    for i in range(19):
        src = pick - (L.E[i, 0] + nx * (L.E[i, 1] + ny * L.E[i, 2]))
        fs = L.collide(o.f[:, src], f_ib[src], c["tau"])
        worst_ib = max(worst_ib, float(np.abs(g1[i, pick] - (fs[i] - L.W[i])).max()))
    # Zou-He faces
    face_err = {}
    for face in range(6):
        if g.faces[face].kind != 0:
            face_err[face] = _face_slab_check(g, face, c["tau"], g1)
    print(f"full-size one step: vertices {dx:.2e}, velocities {dv:.2e}, shell populations {worst_ib:.2e} "
          f"({len(pick)} nodes), faces {face_err}")
    assert dx <= 1e-6 and dv <= 1e-6, (dx, dv)
    assert worst_ib <= 2e-7, worst_ib
    assert sum(nf for nf, _ in face_err.values()) > 1000
    assert all(e <= 2e-7 for _, e in face_err.values()), face_err
