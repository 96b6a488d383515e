"""A stiff capsule meeting the rounded apex of the deformable-capsule
bifurcation (256x96x64, D = 48, junction rounding 8 lu, d = 36 of 2562
vertices, half-angle 30 deg, Ca = 0.005), stepped on the GPU until its
largest edge stretch jumps; the state just before the jump is handed to the
FP64 oracle's coupled operators (Eqs. uLag .. verletPosC), which must give the
same x(t + dt) and vertex velocities as one CUDA step from that state.  The
test prints where the jump happens: the vertex that moves most, its distance
to the nearest solid node, and the oracle's split of its force into probe
pressure, probe viscous stress, stretching, bending and volume terms."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import lattice as L
from oracle import membrane as Mb
from oracle import sim
from paper_2207_06043_gb300 import workloads as W

pytestmark = pytest.mark.gpu

START = 6250          # steps run in one call before stepping one by one
LIMIT = 7000


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.zeros(1, device="cuda")


def _wall_distance(g, x):
    """Distance from x to the nearest solid-node centre within 6 lu (inf if
    none)."""
    nx, ny, nz = g.nx, g.ny, g.nz
    c = np.floor(x).astype(int)
    r = np.arange(-6, 7)
    X, Y, Z = np.meshgrid(c[0] + r, c[1] + r, c[2] + r, indexing="ij")
    ok = (X >= 0) & (X < nx) & (Y >= 0) & (Y < ny) & (Z >= 0) & (Z < nz)
    X, Y, Z = X[ok], Y[ok], Z[ok]
    solid = g.tag[X + nx * (Y + ny * Z)] != 0
    if not solid.any():
        return np.inf
    d = np.sqrt((X[solid] - x[0]) ** 2 + (Y[solid] - x[1]) ** 2 + (Z[solid] - x[2]) ** 2)
    return float(d.min())


def test_apex_contact_step_matches_the_oracle():
    c = W.deformable_capsule(30.0, 0.005)
    g = c["geometry"]
    cap = c["capsules"][0]
    nv = len(cap["verts"])
    s = W.make_solver(c)
    done, _ = s.step(START, allow_damage=True)
    assert done == START
    hist = []
    prev_blob, prev_stretch = None, s.read_capsules(1)[0]["max_stretch"]
    t = START
    jump = None
    while t < LIMIT:
        blob = s.save_state()
        done, _ = s.step(1, allow_damage=True)
        t += 1
        st = s.read_capsules(1)[0]
        hist.append((t, st["max_stretch"]))
        if done == 0 or st["max_stretch"] - prev_stretch > 0.05 or st["max_stretch"] >= 2.0:
            jump = (t, blob, prev_blob)
            break
        prev_blob, prev_stretch = blob, st["max_stretch"]
    print("max stretch, last steps:", [(a, round(b, 4)) for a, b in hist[-8:]])
    if jump is None:
        s.close()
        pytest.skip(f"no jump of the largest stretch before step {LIMIT}")
    t_jump, blob, _ = jump
    # the pre-step state of the jump, then one CUDA step from it
    s.load_state(blob)
    g0 = s.read_populations()
    st0 = s.read_capsule_state(0, nv)
    s.step(1, allow_damage=True)
    st1 = s.read_capsule_state(0, nv)
    s.close()
    lat = SimpleNamespace(nx=g.nx, ny=g.ny, nz=g.nz, N=g.n_nodes, tau=c["tau"], periodic=g.periodic,
                          fluid=g.tag == 0)
    o = sim.Simulation.__new__(sim.Simulation)
    o.lat, o.u_max, o.t, o.damaged, o.last = lat, c["u_max"], 0, False, {}
    o.f = g0.astype(np.float64) + L.W[:, None]
    b = sim.Body(cap["verts"], cap["tris"], cap["params"], c["tau"], cap.get("vel0"))
    b.x, b.x_prev, b.vel = st0["x"].copy(), st0["x_prev"].copy(), st0["vel"].copy()
    o.bodies = [b]
    _, per = o.ib_force()
    Fs = o.structure(o.f, per)
    x0 = st0["x"]
    o.update(o.f, per, Fs)
    dx = float(np.abs(b.x - st1["x"]).max())
    dv = float(np.abs(b.vel - st1["vel"]).max())
    # where it happens
    move = np.linalg.norm(st1["x"] - x0, axis=1)
    k = int(np.argmax(move))
    Av, nrm = per[0]["Av"], per[0]["nrm"]
    Fp, Ft = Mb.hydrodynamic_forces(lat, o.f, x0, Av, nrm)
    V = Mb.diagnostics(x0, b.tris)["volume"]
    Fst = Mb.stretch_forces(x0, b.rest)
    Fb = Mb.bending_forces(x0, b.rest)
    Fv = Mb.volume_forces(x0, b.rest, V, Av, nrm)
    print(f"jump at step {t_jump}: vertex {k} moves {move[k]:.3e} lu (median {np.median(move):.3e}); "
          f"x {np.round(x0[k], 3).tolist()}, n {np.round(nrm[k], 3).tolist()}, "
          f"wall distance {_wall_distance(g, x0[k]):.3f}, probe+ wall distance "
          f"{_wall_distance(g, x0[k] + 1.2 * nrm[k]):.3f}")
    print(f"  U {np.round(per[0]['U'][k], 5).tolist()}; forces: pressure {np.round(Fp[k], 5).tolist()}, "
          f"viscous {np.round(Ft[k], 5).tolist()}, stretch {np.round(Fst[k], 5).tolist()}, "
          f"bending {np.round(Fb[k], 5).tolist()}, volume {np.round(Fv[k], 5).tolist()}; m_v {b.rest.mv:.4f}")
    st = per[0]["stencil"]
    print(f"  marker stencil of the vertex: {int((st.weight[k] > 0).sum())} fluid support nodes, "
          f"sum |phi| {np.abs(st.phi[k]).sum():.3f} (a support wholly in the fluid: "
          f"{np.median(np.abs(st.phi).sum(axis=1)):.3f} median over the vertices)")
    print(f"  CUDA vs oracle from the same state: x {dx:.2e}, velocity {dv:.2e}")
    assert dx <= 1e-5 * max(1.0, move[k]) and dv <= 1e-5 * max(1.0, move[k]), (dx, dv)


def test_apex_contact_window_against_the_oracle():
    """The 40 steps before the jump, from the GPU state, stepped by both
    paths: the growth of the fluid speed near the tip and of the largest edge
    stretch must be the same in the FP64 oracle (it is the method's, not the
    kernels'); the per-step largest stretch agrees within 1e-3 until the
    jump and both paths jump at the same step."""
    from helpers import oracle_for
    c = W.deformable_capsule(30.0, 0.005)
    cap = c["capsules"][0]
    nv = len(cap["verts"])
    s = W.make_solver(c)
    s.step(START, allow_damage=True)
    start = s.save_state()
    t = START
    hist = []
    while t < LIMIT:
        done, _ = s.step(1, allow_damage=True)
        t += 1
        hist.append(s.read_capsules(1)[0]["max_stretch"])
        if done == 0 or hist[-1] >= 2.0 or (len(hist) > 1 and hist[-1] - hist[-2] > 0.05):
            break
    if t >= LIMIT:
        s.close()
        pytest.skip("no jump")
    t_jump = t
    w0 = t_jump - 40
    s.load_state(start)
    s.step(w0 - START, allow_damage=True)
    g0 = s.read_populations()
    st0 = s.read_capsule_state(0, nv)
    gpu = []
    for _ in range(41):
        done, _ = s.step(1, allow_damage=True)
        st = s.read_capsules(1)[0]
        _, u = s.read_fields()
        gpu.append((st["max_stretch"], float(np.linalg.norm(u, axis=1).max())))
        if done == 0:
            break
    s.close()
    lat, o = oracle_for(c, f0=g0.astype(np.float64) + L.W[:, None])
    b = o.bodies[0]
    b.x, b.x_prev, b.vel = st0["x"].copy(), st0["x_prev"].copy(), st0["vel"].copy()
    orc = []
    for _ in range(len(gpu)):
        o.step(1)
        _, uo = lat.macroscopic(o.f)
        orc.append((Mb.max_stretch(b.x, b.rest), float(np.linalg.norm(uo[lat.fluid], axis=1).max())))
    for k, (a, r) in enumerate(zip(gpu, orc)):
        print(f"step {w0 + k + 1}: max stretch {a[0]:.5f} / {r[0]:.5f}, max |u| {a[1]:.4e} / {r[1]:.4e}")
    jump_g = next((k for k, a in enumerate(gpu) if a[0] >= 2.0), None)
    jump_o = next((k for k, r in enumerate(orc) if r[0] >= 2.0), None)
    assert jump_g is not None and jump_o is not None, (jump_g, jump_o)
    assert abs(jump_g - jump_o) <= 1, (jump_g, jump_o)
    for a, r in zip(gpu[:min(jump_g, jump_o)], orc):
        assert abs(a[0] - r[0]) <= 1e-3 * r[0], (a, r)
