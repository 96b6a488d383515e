"""A stiff capsule carried through the rounded apex of the deformable-capsule
bifurcation (256x96x64, D = 48, junction rounding 8 lu, d = 36 of 2562
vertices, half-angle 30 deg, Ca = 0.005).  With solid support nodes dropped
from the MLS fits, the direct forcing near the wall amplified the fluid
velocity by about a third per step (0.021 to above 0.5 lu per step in 12
steps near step 6380, in the FP64 oracle as in the CUDA path) and threw a
vertex a lattice spacing in one step; with the wall's state in the fits
(Reading M4) the flow stays bounded.  The tests find the step of closest
approach to the wall and check there: the largest edge stretch never jumps,
one CUDA step from that state matches the oracle's coupled operators (Eqs.
uLag .. verletPosC), and a 40-step window of both paths agrees step by
step."""
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import lattice as L
from oracle import membrane as Mb
from oracle import sim
from paper_2207_06043_gb300 import workloads as W

pytestmark = pytest.mark.gpu

START = 6000          # the search for the closest approach starts here
STOP = 8000
CHUNK = 25


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


def _closest_approach(s, g, nv):
    """Step from START to STOP in chunks, return (step, distance, state) of
    the chunk boundary where a vertex is nearest a solid node, and the
    largest growth of the largest edge stretch over one chunk."""
    s.step(START, allow_damage=True)
    best = (None, np.inf, None)
    prev = s.read_capsules(1)[0]["max_stretch"]
    worst = 0.0
    for t in range(START, STOP, CHUNK):
        x = s.read_capsule(0, with_verts=True)["verts"]
        front = x[np.argsort(x[:, 0])[-300:]]
        dist = min(_wall_distance(g, p) for p in front)
        if dist < best[1]:
            best = (t, dist, s.save_state())
        done, _ = s.step(CHUNK, allow_damage=True)
        assert done == CHUNK, t
        st = s.read_capsules(1)[0]["max_stretch"]
        worst = max(worst, st - prev)
        prev = st
    return best, worst


def test_apex_contact_step_matches_the_oracle():
    c = W.deformable_capsule(30.0, 0.005)
    g = c["geometry"]
    cap = c["capsules"][0]
    nv = len(cap["verts"])
    s = W.make_solver(c)
    (t_c, dist, blob), worst = _closest_approach(s, g, nv)
    print(f"closest approach at step {t_c}: a vertex {dist:.3f} lu from a solid node; largest growth of the "
          f"max stretch over {CHUNK} steps {worst:.2e}")
    assert worst < 0.05, worst
    # one CUDA step from the state of closest approach
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
    o.update(o.f, per, Fs)
    dx = float(np.abs(b.x - st1["x"]).max())
    dv = float(np.abs(b.vel - st1["vel"]).max())
    st = per[0]["stencil"]
    solid = (~lat.fluid[st.nodes]).any(axis=1)
    print(f"step {t_c + 1}: {int(solid.sum())} marker stencils with solid support nodes; "
          f"CUDA vs oracle: x {dx:.2e}, velocity {dv:.2e}")
    assert solid.sum() > 0
    assert dx <= 1e-5 and dv <= 1e-5, (dx, dv)


def test_apex_contact_window_against_the_oracle():
    """40 steps around the closest approach, from the GPU state, by both
    paths: per step the largest stretch and the largest fluid speed agree
    within 1e-3 relative, and the speed stays below 1.5 times its start."""
    from helpers import oracle_for
    c = W.deformable_capsule(30.0, 0.005)
    cap = c["capsules"][0]
    nv = len(cap["verts"])
    s = W.make_solver(c)
    (t_c, _, _), _ = _closest_approach(s, c["geometry"], nv)
    s.close()
    s = W.make_solver(c)
    w0 = max(t_c - 20, 1)
    s.step(w0, allow_damage=True)
    g0 = s.read_populations()
    st0 = s.read_capsule_state(0, nv)
    gpu = []
    for _ in range(40):
        done, _ = s.step(1, allow_damage=True)
        assert done == 1
        st = s.read_capsules(1)[0]
        _, u = s.read_fields()
        gpu.append((st["max_stretch"], float(np.linalg.norm(u, axis=1).max())))
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
    assert max(r[1] for r in orc) < 1.5 * orc[0][1]
    for a, r in zip(gpu, orc):
        assert abs(a[0] - r[0]) <= 1e-3 * r[0] and abs(a[1] - r[1]) <= 1e-3 * r[1], (a, r)
