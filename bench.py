"""Throughput benchmark of the coupled LB / dynamic-IB time step on GB300.

One bench step = one full time step of the method (IB pre-pass, collide +
stream with Zou-He faces, BFL wall fill, membrane / probe forces, repulsion,
Verlet update, damage check) on the throughput workload: a 512x192x128 duct
splitting twice (D = 96, half-angles 40 deg) carrying 64 deformable capsules
of 2562 vertices.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|f16|bf16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a sample
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline (fwd, adjoint, batched); error vs FP64 oracle"
BYTES_PER_UPDATE = {"f32": 152, "f16": 76, "bf16": 76}
# DRAM read + write of one FP32 lattice-kernel launch on the throughput
# workload, from an ncu capture of two launches of the timed region (kept
# with the profile summaries); valid only for the kernel as captured and that
# workload.
LBM_TRAFFIC_BYTES = {("throughput", "f32"): 623.4e6}
CPU_SAMPLE_X = 64          # x-slab of the workload the oracle runs on (cpu_baseline)
REF_SAMPLE_X = 16          # thinner slab per step of the reference arm
WORKLOADS = {
    # the throughput configuration (12.6 M nodes, 64 capsules)
    "throughput": dict(),
    # a smaller instance of the same family for profiler captures (~4 M nodes)
    "small": dict(n_capsules=32, nx=320, ny=128, nz=96, D=64.0, d=16.0, nv=2562),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def fluid_updates(case):
    return int(np.count_nonzero(case["geometry"].tag == 0))


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank returns it)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(fluid_nodes_per_rank, steps, ms, world):
    """Fluid-node updates of all ranks (weak scaling: each rank its own
    replica of the workload) per second of the slowest rank, in millions."""
    return world * fluid_nodes_per_rank * steps / (ms * 1e-3) / 1e6


def cpu_sample_case(case, x1=CPU_SAMPLE_X):
    """The x-slab [0, x1) of the workload with the capsules lying inside it."""
    from paper_2207_06043_gb300 import geometry as G
    g = G.crop_x(case["geometry"], x1)
    caps = [c for c in case["capsules"] if c["verts"][:, 0].max() < x1 - 6]
    return dict(case, geometry=g, capsules=caps)


def run_oracle(case, steps, warmup=0):
    """Time the FP64 oracle as it stands on `case` (host cores)."""
    from oracle import lattice as L
    from oracle import sim
    g = case["geometry"]
    lat = L.Lattice(g.nx, g.ny, g.nz, case["tau"], g.tag, g.links, g.faces, g.periodic)
    o = sim.Simulation(lat, u_max=case["u_max"])
    for c in case["capsules"]:
        o.add_body(c["verts"], c["tris"], c["params"], c.get("vel0"))
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return dt, int(np.count_nonzero(lat.fluid))


def cpu_threads():
    """The oracle's array work is numpy element-wise code: one host thread."""
    return 1


def reference_arm(args, rank):
    """--impl reference: the FP64 oracle, as it stands, on a bounded sample."""
    from paper_2207_06043_gb300 import workloads as W
    if rank != 0:
        return
    case = W.throughput_case(**WORKLOADS[args.workload])
    sample = cpu_sample_case(case, REF_SAMPLE_X)
    dt, nf = run_oracle(sample, args.steps, args.warmup)
    mlups = nf * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": case["name"], "sample": f"x-slab [0,{REF_SAMPLE_X}) with "
                       f"{len(sample['capsules'])} capsules", "fluid_nodes": nf},
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"x-slab [0,{REF_SAMPLE_X}) of the workload ({nf} fluid nodes, "
                                       f"{len(sample['capsules'])} capsules), {args.steps} steps"},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="throughput", choices=sorted(WORKLOADS) + ["sweep"])
    ap.add_argument("--members", type=int, default=64, help="lattices of the batched sweep workload")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the 16-bit storage side measurements")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-ckpt", type=int, default=2000)
    ap.add_argument("--threads", type=int, default=128)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.workload == "sweep":
        sweep_bench(args, rank, world, local)
        return

    import torch
    torch.cuda.set_device(local)
    torch.zeros(1, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2207_06043_gb300 import workloads as W

    case = W.throughput_case(**WORKLOADS[args.workload])
    nf = fluid_updates(case)
    s = W.make_solver(case, storage=args.storage)
    s.set_launch(args.threads, args.blocks_per_sm)
    s.step(args.warmup)

    # timed region: per-kernel CUDA events recorded on the library's stream
    s.enable_timing(True)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        done, _ = s.step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    kt = s.kernel_times()
    s.enable_timing(False)
    # graph replay (production mode) over the same number of steps
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    s.step(args.steps)
    g1.record(stream)
    torch.cuda.synchronize()
    ms_graph = g0.elapsed_time(g1)
    ms_best = max_over_ranks(min(ms, ms_graph), dist, "cuda")
    value = whole_job_mlups(nf, args.steps, ms_best, world)
    launches = s.kernels_per_step() * args.steps

    bpu = BYTES_PER_UPDATE[args.storage]
    peak, peak_kind = load_peaks()
    lbm_ms = kt["lattice"] / args.steps
    achieved = bpu * nf / (lbm_ms * 1e-3) / 1e9
    traffic = LBM_TRAFFIC_BYTES.get((args.workload, args.storage))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of two launches"
                               if traffic else None), "kernel": "k_lbm (fused collide+stream, AA pattern)",
            "peak_source": f"{peak_kind} hbm_gbs", "ms_per_launch": lbm_ms,
            "algorithmic_bytes_per_launch": bpu * nf}
    s.close()

    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_best / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
           "config": {"workload": case["name"], "fluid_nodes": nf, "box_nodes": case["geometry"].n_nodes,
                      "capsules": len(case["capsules"]), "markers": sum(len(c["verts"]) for c in case["capsules"]),
                      "storage": args.storage, "l2": "inputs larger than L2 (distributions ~1 GB)",
                      "parallelism": "replicas" if world > 1 else "1 GPU",
                      "launch": {"threads": args.threads, "blocks_per_sm": args.blocks_per_sm}},
           "roofline": roof,
           "kernel_ms_per_step": {k: v / args.steps for k, v in kt.items()},
           "ms_per_step_timed_events": ms / args.steps, "ms_per_step_graph": ms_graph / args.steps,
           "clocks": clk.summary(),
           "gpu_launches": launches}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_run(case, args)
    if rank == 0 and not args.no_adjoint:
        out["adjoint"] = adjoint_measure(args, case)
    if rank == 0 and not args.no_variants and args.storage == "f32":
        out["storage_variants"] = storage_variants(case, nf)
    if rank == 0 and not args.no_cpu:
        sample = cpu_sample_case(case)
        dt, nfs = run_oracle(sample, args.cpu_steps)
        out["cpu_baseline"] = {"value": nfs * args.cpu_steps / dt / 1e6, "unit": "MLUPS", "cores": cpu_threads(),
                               "kind": "oracle",
                               "sample": f"x-slab [0,{CPU_SAMPLE_X}) of the workload ({nfs} fluid nodes, "
                                         f"{len(sample['capsules'])} capsules), {args.cpu_steps} steps"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def storage_variants(case, nf, steps=100):
    """The same workload with f - w stored as FP16 (scaled by 2^12) or BF16,
    FP32 arithmetic: whole-step MLUPS (graph replay) and the lattice kernel's
    fraction of the HBM roofline at 76 B per fluid-node update."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    peak, kind = load_peaks()
    out = {}
    stream = torch.cuda.current_stream()
    for st in ("f16", "bf16"):
        s = W.make_solver(case, storage=st)
        s.step(5)
        s.enable_timing(True)
        s.step(steps)
        lat = s.kernel_times()["lattice"] / steps
        s.enable_timing(False)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        s.close()
        ach = BYTES_PER_UPDATE[st] * nf / (lat * 1e-3) / 1e9
        out[st] = {"value": nf / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms, "steps": steps,
                   "lattice_ms": lat, "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                                   "frac": ach / peak, "peak_source": f"{kind} hbm_gbs"}}
    return out


def _adjoint_run(c, n, K, lo, hi):
    """Time n plain forward steps and one ibl_adjoint call of n steps on the
    lattice of case c (no capsules), each on its own context; the adjoint is
    timed on its second call (the first allocates its buffers and captures
    its graphs)."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    fwd = W.make_solver(c)
    adj = W.make_solver(c)
    fwd.step(10)
    adj.step(10)
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    e[0].record(stream)
    fwd.step(n)
    e[1].record(stream)
    adj.adjoint(n, lo, hi, (1.0, 0.0, 0.0), ckpt_every=K)     # allocates the buffers, captures the graphs
    torch.cuda.synchronize()
    e[2].record(stream)
    J, gs, gr = adj.adjoint(n, lo, hi, (1.0, 0.0, 0.0), ckpt_every=K)
    e[3].record(stream)
    torch.cuda.synchronize()
    ms_f, ms_a = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    fwd.close()
    adj.close()
    nf = fluid_updates(c)
    return {"fluid_nodes": nf, "steps": n, "ckpt_every": K, "ms_forward": ms_f, "ms_adjoint_call": ms_a,
            "cost_vs_forward": ms_a / ms_f, "mlups_adjoint": nf * n / (ms_a * 1e-3) / 1e6,
            "J": J, "dJ_du_max": gs / c["u_max"], "dJ_dr_j": gr}


def adjoint_measure(args, case):
    """The discrete adjoint (ibl_adjoint) against the same number of plain
    forward steps, on (a) the adjoint workload's lattice (192x64x48
    bifurcation, junction radius 4 lu, 2000 steps) and (b) the throughput
    workload's lattice (12.6 M nodes, 100 steps), each with its whole tape in
    HBM (one segment: no recompute; about 20 GB each),
    both without capsules: the adjoint covers the lattice step.  J = sum of
    u_x over the upper half of the region just past the junction (a), of the
    inlet region (b)."""
    from paper_2207_06043_gb300 import workloads as W
    out = {"note": "each timed call runs the forward sweep writing the tape and the reverse sweep (one "
                   "segment: nothing recomputed); its buffers and graphs come from a first, untimed call"}
    ca = dict(W.adjoint_case(), capsules=[])
    g = ca["geometry"]
    xj = int(g.info["x_junction"])
    r = _adjoint_run(ca, args.adjoint_steps, args.adjoint_ckpt, (xj, int(g.info["yc"]), 0),
                     (min(g.nx, xj + 24), g.ny, g.nz))
    out["adjoint_workload"] = dict(r, workload="bifurcation 192x64x48, D 36, 45 deg, junction radius 4 lu, no capsule")
    ct = dict(case, capsules=[])
    g = ct["geometry"]
    xj = int(g.info["x_junction"])
    r = _adjoint_run(ct, 100, 100, (4, int(g.info["yc"]), 0), (52, g.ny, g.nz))
    bpu = 168 + 168            # forward step writing the tape, adjoint step (B per fluid node and step)
    peak, kind = load_peaks()
    ach = bpu * r["fluid_nodes"] * r["steps"] / (r["ms_adjoint_call"] * 1e-3) / 1e9
    out["throughput_lattice"] = dict(r, workload="throughput lattice 512x192x128 without capsules",
                                     roofline={"bound": "hbm", "algorithmic_bytes_per_node_step": bpu,
                                               "achieved": ach, "peak": peak, "unit": "GB/s",
                                               "frac": ach / peak, "peak_source": f"{kind} hbm_gbs"})
    return out


def _sweep_member(k):
    from paper_2207_06043_gb300 import workloads as W
    c = W.sweep_member(k)
    c["geometry"].sdf = None          # closures do not cross process boundaries
    return c


def sweep_bench(args, rank, world, local):
    """Batched sweep: the members of the sweep workload stepped together as one
    context (one launch per kernel per step for all lattices, CUDA graphs),
    launch shape chosen by the library's autotuner.  MLUPS counts the fluid
    nodes of the members that are still running (a capsule that breaks stops
    its lattice, as the damage rule says)."""
    import multiprocessing as mp
    # inputs are generated before CUDA starts, in spawned workers
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        members = pool.map(_sweep_member, range(args.members))
    import torch
    torch.cuda.set_device(local)
    torch.zeros(1, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2207_06043_gb300 import binding
    from paper_2207_06043_gb300 import workloads as W
    nf = [fluid_updates(c) for c in members]
    ens = binding.ensemble([W.make_solver(c) for c in members])
    ens.step(args.warmup, allow_damage=True)
    thr, bps, _ = ens.autotune(4)
    n_m = len(members)

    def steps_done():
        return [ens.member_steps(m) for m in range(n_m)]

    stream = torch.cuda.current_stream()
    # lattice-kernel time per step from a timing-mode pass
    ens.enable_timing(True)
    c0 = steps_done()
    ens.step(args.steps, allow_damage=True)
    c1 = steps_done()
    kt = ens.kernel_times()
    ens.enable_timing(False)
    upd_timing = sum(nf[m] * (c1[m] - c0[m]) for m in range(n_m))
    # timed region: graph replay
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        ens.step(args.steps, allow_damage=True)
        e1.record(stream)
        torch.cuda.synchronize()
    c2 = steps_done()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    upd = sum(nf[m] * (c2[m] - c1[m]) for m in range(n_m))
    value = world * upd / (ms * 1e-3) / 1e6
    bpu = BYTES_PER_UPDATE["f32"]
    peak, peak_kind = load_peaks()
    achieved = bpu * upd_timing / (kt["lattice"] * 1e-3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batched sweep: {n_m} bifurcations of uneven size, one capsule each",
                      "fluid_nodes": int(sum(nf)), "box_nodes": int(sum(c["geometry"].n_nodes for c in members)),
                      "running_members": int(sum(1 for m in range(n_m) if c2[m] - c1[m] == args.steps)),
                      "l2": "inputs larger than L2", "launch": {"threads": thr, "blocks_per_sm": bps,
                                                                "chosen_by": "ibl_autotune"}},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "k_lbm (all members in one launch)", "peak_source": f"{peak_kind} hbm_gbs"},
           "kernel_ms_per_step": {k: v / args.steps for k, v in kt.items()},
           "clocks": clk.summary(), "gpu_launches": ens.kernels_per_step() * args.steps}
    ens.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def e2e_run(case, args):
    """The same metric through the public API from host buffers: context set-up
    (every input array copied host -> device), the time steps, capsule
    diagnostics read back every 100 steps and the fields read at the end, all
    inside the timed region."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    g = case["geometry"]
    nf = fluid_updates(case)
    h2d = g.tag.nbytes + g.links.nbytes + sum(f.velocity.nbytes for f in g.faces if f.velocity is not None)
    h2d += sum(c["verts"].nbytes + c["tris"].nbytes for c in case["capsules"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = W.make_solver(case, storage=args.storage)
    s.set_launch(args.threads, args.blocks_per_sm)
    d2h = 0
    left = args.steps
    while left > 0:
        k = min(100, left)
        s.step(k)
        left -= k
        for cid in range(len(case["capsules"])):
            s.read_capsule(cid)
            d2h += 2 * 3 * 8 * len(case["capsules"][cid]["verts"])
    rho, u = s.read_fields()
    d2h += rho.nbytes + u.nbytes
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return {"value": nf * args.steps / dt / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
            "d2h_bytes_per_step": d2h / args.steps,
            "note": "includes context set-up from host arrays (topology, uploads, initial state)"}


if __name__ == "__main__":
    main()
