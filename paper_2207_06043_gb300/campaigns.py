"""Runner of the paper's experiment campaigns (single capsules, trains of
three, mixed rigid / soft trains; Section "Results and discussion") through
the library: the cases are stepped together as one batched context, each
member optionally started from the stationary flow of its geometry without
capsules (the paper's initial condition), and every capsule's FP64
diagnostics are read every `every` steps.  Argument marshalling and
bookkeeping only: every step runs in the CUDA library."""
from __future__ import annotations

import numpy as np

from . import binding
from . import workloads as W


def stationary_flow(case, steps):
    """(rho, u) after `steps` steps of the case's geometry without capsules."""
    s = W.make_solver(dict(case, capsules=[]))
    s.step(int(steps))
    rho, u = s.read_fields()
    s.close()
    return rho, u


def run(cases, steps, every=500, warm_steps=0):
    """Step the cases together; returns, per case, per capsule, the arrays
    t (steps), centroid (n, 3), dS, taylor_D, max_stretch and velocity (n, 3),
    plus the steps each member completed (a damaged capsule stops its
    member, as the paper's damage rule says)."""
    solvers = []
    for c in cases:
        s = W.make_solver(c)
        if warm_steps:
            rho, u = stationary_flow(c, warm_steps)
            s.init_equilibrium(rho, u)
        solvers.append(s)
    ens = binding.ensemble(solvers)
    n_caps = [len(c["capsules"]) for c in cases]
    rec = [[dict(t=[], centroid=[], dS=[], taylor_D=[], max_stretch=[], velocity=[]) for _ in range(n)]
           for n in n_caps]
    done = 0
    while done < steps:
        k = min(every, steps - done)
        ens.step(k, allow_damage=True)
        done += k
        for m, n in enumerate(n_caps):
            if n == 0:
                continue
            t = ens.member_steps(m)
            for ci, st in enumerate(ens.read_capsules(n, member=m)):
                r = rec[m][ci]
                if r["t"] and r["t"][-1] == t:
                    continue          # the member has stopped
                r["t"].append(t)
                r["centroid"].append(st["centroid"])
                r["dS"].append(st["dS"])
                r["taylor_D"].append(st["taylor_D"])
                r["max_stretch"].append(st["max_stretch"])
                r["velocity"].append(st["velocity"])
    out = []
    for m, c in enumerate(cases):
        caps = []
        for r in rec[m]:
            caps.append({k: np.asarray(v) for k, v in r.items()})
        out.append(dict(name=c["name"], steps_done=ens.member_steps(m), capsules=caps))
    ens.close()
    return out


def summary(case, result):
    """Per capsule: the largest relative stretching dS, the time of it in
    units of d / u_max, and the streamwise position of the centroid then,
    in units of d (the quantities of the paper's stretching figures)."""
    d = case["geometry"].info["D"]
    u = case["u_max"]
    rows = []
    for r in result["capsules"]:
        if len(r["t"]) == 0:
            rows.append(dict(dS_max=None))
            continue
        i = int(np.argmax(r["dS"]))
        rows.append(dict(dS_max=float(r["dS"][i]), t_star=float(r["t"][i] * u / d),
                         x_over_d=float(r["centroid"][i][0] / d), max_stretch=float(r["max_stretch"].max()),
                         damaged=bool(r["max_stretch"].max() >= 2.0)))
    return rows
