"""Shared helpers: build the oracle and the CUDA path from the same inputs."""
import numpy as np

from oracle import lattice as L
from oracle import sim


def oracle_for(case, f0=None):
    g = case["geometry"]
    lat = L.Lattice(g.nx, g.ny, g.nz, case["tau"], g.tag, g.links, g.faces, g.periodic,
                    body_force=case.get("body_force", (0.0, 0.0, 0.0)))
    o = sim.Simulation(lat, f0=f0, u_max=case["u_max"])
    for c in case["capsules"]:
        o.add_body(c["verts"], c["tris"], c["params"], c.get("vel0"))
    return lat, o


def gpu_for(case, storage="f32"):
    from paper_2207_06043_gb300.binding import Solver
    g = case["geometry"]
    s = Solver.from_geometry(g, case["tau"], storage=storage, body_force=case.get("body_force", (0.0, 0.0, 0.0)),
                             u_max=case["u_max"])
    for c in case["capsules"]:
        s.add_capsule(c["verts"], c["tris"], vel0=c.get("vel0"), **c["params"])
    return s


def rel_l2(a, b, mask=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(geometry, tau=0.8, u_max=0.02, capsules=(), body_force=(0.0, 0.0, 0.0)):
    return dict(geometry=geometry, tau=tau, u_max=u_max, capsules=list(capsules), body_force=body_force)
