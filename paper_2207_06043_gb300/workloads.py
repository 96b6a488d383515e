"""Seeded synthetic workloads: square-duct bifurcations with capsules, sized as
the standard cases of the solver (the paper's set-up of Section "Computational
set-up and boundary conditions" re-cast on square ducts).  Each builder returns
a plain dict of inputs (geometry, tau, capsules, steps) that both the CUDA
library and the FP64 oracle can consume; nothing here computes the method.
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry as G
from . import meshes as Ms

SEED = 2207
TAU = 0.8
NU = (TAU - 0.5) / 3.0


def _capsule(verts, tris, rigid=False, Ca=0.01, Eb=0.001, kv=1.0, density_ratio=1.1, u_ref=0.02, vel0=None):
    return dict(verts=np.asarray(verts, np.float64), tris=np.asarray(tris, np.int32),
                params=dict(Ca=Ca, Eb=Eb, kv=kv, density_ratio=density_ratio, u_ref=u_ref, rigid=int(rigid)),
                vel0=vel0)


def bifurcation_small(seed=SEED):
    """96x32x32 Y-bifurcation, D = 24, half-angle 45 deg, sharp junction,
    Poiseuille inlet u_max = 0.02, pressure outlets; one rigid sphere d = 12
    (642-vertex icosphere) released at x = 20, 2 lu off-axis; 500 steps."""
    g = G.bifurcation(96, 32, 32, 24.0, 45.0, 0.0, u_max=0.02)
    rng = Ms.SplitMix64(seed)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    c = (20.0, g.info["yc"] + 2.0 * math.cos(phi), g.info["zc"] + 2.0 * math.sin(phi))
    V, T = Ms.sphere_mesh(642, 12.0, c, rng)
    return dict(name="bifurcation 96x32x32, rigid sphere d=12 (642 v), 500 steps", geometry=g, tau=TAU,
                u_max=0.02, capsules=[_capsule(V, T, rigid=True)], steps=500)


def deformable_capsule(half_angle=45.0, Ca=0.01, seed=SEED):
    """256x96x64 bifurcation, D = 48, junction rounding 8 lu, one capsule
    d = 36 (2562 v), Re = u_max D / nu = 10; 20k steps."""
    D = 48.0
    u_max = 10.0 * NU / D
    g = G.bifurcation(256, 96, 64, D, half_angle, 8.0, u_max=u_max)
    rng = Ms.SplitMix64(seed)
    c = (18.0 + 4.0, g.info["yc"], g.info["zc"])
    V, T = Ms.sphere_mesh(2562, 36.0, c, rng)
    return dict(name=f"bifurcation 256x96x64, capsule d=36 (2562 v), half-angle {half_angle}, Ca {Ca}",
                geometry=g, tau=TAU, u_max=u_max, capsules=[_capsule(V, T, Ca=Ca, u_ref=u_max)], steps=20000)


def adjoint_case(seed=SEED):
    """192x64x48 bifurcation, D = 36, half-angle 45, junction rounding 4 lu
    (with dq/dr_j per link), capsule d = 27 (2562 v), Ca = 0.01; 2000 steps."""
    g = G.bifurcation(192, 64, 48, 36.0, 45.0, 4.0, u_max=0.02, with_dq=True)
    rng = Ms.SplitMix64(seed)
    V, T = Ms.sphere_mesh(2562, 27.0, (13.5 + 4.0, g.info["yc"], g.info["zc"]), rng)
    return dict(name="bifurcation 192x64x48, capsule d=27 (2562 v), Ca 0.01", geometry=g, tau=TAU, u_max=0.02,
                capsules=[_capsule(V, T, Ca=0.01)], steps=2000)


def throughput_case(seed=SEED, n_capsules=64, nx=512, ny=192, nz=128, D=96.0, d=24.0, nv=2562):
    """512x192x128 (12.6 M nodes) duct splitting twice (D = 96 -> 68 -> 48,
    half-angles 40 deg), 64 deformable capsules d = 24 (2562 v each) at seeded
    non-overlapping positions in the inlet third, Ca = 0.02, Re = 20; 10k steps.

    Placement: the sites of a two-layer packing (3x3 grid at 34 lu pitch, then
    a 2x2 grid offset by half a pitch, layers 13 lu apart; every pair of
    centres at least d + 2 apart, 2 lu from the walls) restricted to the inlet
    third; n_capsules sites are drawn without replacement by SplitMix64 and
    each mesh gets a random rotation."""
    u_max = 20.0 * NU / D
    g = G.bifurcation(nx, ny, nz, D, 40.0, 0.0, u_max=u_max, levels=2, x_junction=0.4 * nx)
    yc, zc = g.info["yc"], g.info["zc"]
    lim = D / 2 - d / 2 - 2.0
    sites = []
    x = d / 2 + 2.0
    layer = 0
    while x <= nx / 3.0 - d / 2 - 2.0:
        if layer % 2 == 0:
            for a in (-lim, 0.0, lim):
                for b in (-lim, 0.0, lim):
                    sites.append((x, yc + a, zc + b))
        else:
            for a in (-lim / 2, lim / 2):
                for b in (-lim / 2, lim / 2):
                    sites.append((x, yc + a, zc + b))
        x += (d + 2.0) / 2.0
        layer += 1
    sites = np.array(sites)
    if len(sites) < n_capsules:
        raise ValueError(f"only {len(sites)} sites for {n_capsules} capsules")
    rng = Ms.SplitMix64(seed)
    order = list(range(len(sites)))
    for i in range(len(order) - 1, 0, -1):   # Fisher-Yates with SplitMix64
        j = rng.randint(0, i)
        order[i], order[j] = order[j], order[i]
    chosen = sites[sorted(order[:n_capsules])]
    caps = []
    for c in chosen:
        V, T = Ms.sphere_mesh(nv, d, c, rng)
        caps.append(_capsule(V, T, Ca=0.02, u_ref=u_max))
    return dict(name=f"duct {nx}x{ny}x{nz} splitting twice (D {D:g}, 40 deg), {n_capsules} capsules d={d:g} ({nv} v)",
                geometry=g, tau=TAU, u_max=u_max, capsules=caps, steps=10000)


def sweep_member(k, seed=SEED):
    """Member k of the batched sweep, drawn from its own SplitMix64 stream
    (seed, k): a bifurcation with dims from 128..384 x 48..128 x 32..96 in
    multiples of 8, half-angle U[20, 80], occlusion U[0.3, 0.9], Ca
    log-U[1e-3, 1e-1], junction rounding U[0, 10]; one capsule (642 v if
    d <= 20 lu else 2562 v) near the inlet, the junction at 0.4 nx or, for a
    long capsule, d + 12 lu from the inlet; 5k steps."""
    rng = Ms.SplitMix64((seed << 20) + k)
    nx = 8 * rng.randint(16, 48)
    ny = 8 * rng.randint(6, 16)
    nz = 8 * rng.randint(4, 12)
    th = rng.uniform(20.0, 80.0)
    occ = rng.uniform(0.3, 0.9)
    Ca = 10.0 ** rng.uniform(-3.0, -1.0)
    rj = rng.uniform(0.0, 10.0)
    D = float(round(0.75 * min(ny, nz)))
    d = occ * D
    u_max = 0.02
    # the junction lies past the capsule's start position (it starts whole
    # inside the main duct, d/2 + 4 from the inlet)
    g = G.bifurcation(nx, ny, nz, D, th, rj, u_max=u_max, x_junction=max(0.4 * nx, d + 12.0))
    nv = 642 if d <= 20.0 else 2562
    c = (d / 2 + 4.0, g.info["yc"], g.info["zc"])
    V, T = Ms.sphere_mesh(nv, d, c, rng)
    return dict(name=f"member {k}: {nx}x{ny}x{nz} th={th:.1f} occ={occ:.2f} Ca={Ca:.4f} rj={rj:.1f}",
                geometry=g, tau=TAU, u_max=u_max, capsules=[_capsule(V, T, Ca=Ca, u_ref=u_max)], steps=5000)


def sweep_case(seed=SEED, n=64):
    """The batched sweep: n independent members (see sweep_member)."""
    return [sweep_member(k, seed) for k in range(n)]


def make_solver(case, storage="f32", stream=None):
    """Library context for a case dict (geometry + capsules)."""
    from .binding import Solver
    g = case["geometry"]
    s = Solver.from_geometry(g, case["tau"], storage=storage, u_max=case["u_max"], stream=stream)
    for c in case["capsules"]:
        s.add_capsule(c["verts"], c["tris"], vel0=c.get("vel0"), **c["params"])
    return s


# ----------------------------------------------------------------------------
# The paper's experiment campaigns (Section "Results and discussion") on its
# circular-duct bifurcation: d = 30 lu, daughters 0.7 d, main duct 6.7 d,
# branches 5 d, tau = 0.75, Eb = 0.001, density ratio 1.1, capsules released
# at 1.16 d from the inlet on the duct axis.  The paper runs at Re = 0.01
# (u_max = 2.8e-5 lu, some 10^7 steps per passage); these builders take Re as
# a parameter (default 1, the Stokes-like regime at a cost of about 10^5
# steps per passage).
# ----------------------------------------------------------------------------
PAPER_D = 30.0
PAPER_TAU = 0.75
PAPER_N_MARKERS = {1.0 / 3.0: 325, 0.5: 485, 2.0 / 3.0: 645, 5.0 / 6.0: 785}


def paper_geometry(half_angle_deg=30.0, smooth=False, Re=1.0):
    nu = (PAPER_TAU - 0.5) / 3.0
    u_max = Re * nu / PAPER_D
    return G.circular_bifurcation(PAPER_D, half_angle_deg, smooth=smooth, u_max=u_max), u_max


def _paper_markers(dp_ratio):
    for k, n in PAPER_N_MARKERS.items():
        if abs(k - dp_ratio) < 1e-9:
            return n
    return int(round(325 + (785 - 325) * (dp_ratio - 1.0 / 3.0) / 0.5))


def paper_single_capsule(half_angle_deg=30.0, smooth=False, dp_ratio=2.0 / 3.0, Ca=0.05, Re=1.0, seed=SEED):
    """One soft capsule of diameter dp_ratio d (n_L markers as the paper lists
    them: 325, 485, 645, 785 for d_p/d = 1/3, 1/2, 2/3, 5/6) released at
    1.16 d from the inlet on the axis."""
    g, u_max = paper_geometry(half_angle_deg, smooth, Re)
    dp = dp_ratio * PAPER_D
    V, T = Ms.sphere_mesh_n(_paper_markers(dp_ratio), dp, (1.16 * PAPER_D, g.info["yc"], g.info["zc"]),
                            Ms.SplitMix64(seed))
    return dict(name=f"paper bifurcation th={half_angle_deg:g} {'smooth' if smooth else 'sharp'}, d_p/d="
                     f"{dp_ratio:.3f}, Ca={Ca:g}, Re={Re:g}",
                geometry=g, tau=PAPER_TAU, u_max=u_max,
                capsules=[_capsule(V, T, Ca=Ca, u_ref=u_max)], steps=int(40 * PAPER_D / u_max))


def paper_train(half_angle_deg=30.0, smooth=False, Ca=0.01, kinds=("soft", "soft", "soft"), Re=1.0, seed=SEED):
    """Three bodies of d_p = 2/3 d in a row along the axis, centres 0.85 d apart,
    the last one (nearest the inlet) at 1.16 d: "soft" capsules (645 markers)
    or "rigid" spheres of diameter d_p / 2 with the same density (325
    markers), listed from the last to the leading one."""
    g, u_max = paper_geometry(half_angle_deg, smooth, Re)
    dp = 2.0 / 3.0 * PAPER_D
    rng = Ms.SplitMix64(seed)
    caps = []
    for k, kind in enumerate(kinds):
        c = ((1.16 + 0.85 * k) * PAPER_D, g.info["yc"], g.info["zc"])
        if kind == "soft":
            V, T = Ms.sphere_mesh_n(645, dp, c, rng)
            caps.append(_capsule(V, T, Ca=Ca, u_ref=u_max))
        else:
            V, T = Ms.sphere_mesh_n(325, 0.5 * dp, c, rng)
            caps.append(_capsule(V, T, rigid=True))
    return dict(name=f"paper bifurcation th={half_angle_deg:g} {'smooth' if smooth else 'sharp'}, train "
                     f"{'/'.join(kinds)}, Ca={Ca:g}, Re={Re:g}",
                geometry=g, tau=PAPER_TAU, u_max=u_max, capsules=caps, steps=int(40 * PAPER_D / u_max))
