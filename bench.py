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
# with the profile summaries), with the hash of the lattice kernel's sources
# (lbm.cu, lbm_device.cuh) it was captured from: any change to them makes the
# figure stale, and the bench then reports null until it is captured again.
LBM_TRAFFIC = {("throughput", "f32"): (633.6e6, "a72606f2c37f77cf")}
LBM_SOURCES = ("lbm.cu", "lbm_device.cuh", "ib.cu")   # ib.cu: the shell pass sets the IB flags the lattice kernel reads
CPU_SAMPLE_X = 64          # x-slab of the workload the oracle runs on (cpu_baseline)
REF_SAMPLE_X = 40          # slab of the reference arm (its first layer of capsules)
PARITY_STEPS = 50          # oracle-parity window on the small bifurcation
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


def lbm_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in LBM_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_06043_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def lbm_traffic(workload, storage):
    """Captured DRAM bytes per lattice-kernel launch, or None when none was
    captured for this workload/storage or the kernel changed since."""
    rec = LBM_TRAFFIC.get((workload, storage))
    if rec is None or rec[1] != lbm_source_hash():
        return None
    return rec[0]


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_worker(args):
    """One oracle process: `steps` timed steps of the sample.  Returns
    (seconds, fluid nodes)."""
    sample, steps = args
    return run_oracle(sample, steps, warmup=0)


def oracle_throughput(sample, steps, procs):
    """Time `procs` independent copies of the oracle on the sample at once, one
    per host core (spawned processes whose numpy runs one thread: the thread
    variables are set before the children import it).  Returns (aggregate
    MLUPS, wall seconds, fluid nodes per copy)."""
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    for k in THREAD_VARS:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, [(sample, steps)] * procs)
            wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    nf = res[0][1]
    slowest = max(r[0] for r in res)
    return procs * nf * steps / slowest / 1e6, wall, nf


def cpu_baseline(case, steps, all_cores=True):
    """The FP64 oracle as it stands on the x-slab sample of the workload: one
    process with one numpy thread, then (all_cores) one independent copy per
    host core at once (throughput; the oracle has no loop parallelism of its
    own)."""
    sample = cpu_sample_case(case)
    sample["geometry"].sdf = None          # closures do not cross process boundaries
    nproc = os.cpu_count() or 1
    mlups1, wall1, nf = oracle_throughput(sample, steps, 1)
    out = {"value": mlups1, "unit": "MLUPS", "cores": 1, "kind": "oracle",
           "sample": f"x-slab [0,{CPU_SAMPLE_X}) of the workload ({nf} fluid nodes, "
                     f"{len(sample['capsules'])} capsules), {steps} step(s) per copy",
           "cpu_model": cpu_model(), "nproc": nproc}
    if all_cores and nproc > 1:
        # each copy holds about 1.5 GB; stay within the available memory
        try:
            avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
            procs = max(1, min(nproc, int(avail // 2.0e9)))
        except (ValueError, OSError):
            procs = nproc
        mlups_n, wall_n, _ = oracle_throughput(sample, steps, procs)
        out["all_cores"] = {"value": mlups_n, "unit": "MLUPS", "cores": procs,
                            "mode": "one independent oracle copy per core, one numpy thread each",
                            "wall_s": wall_n}
    return out


def workload_config(case, storage, world, threads, blocks_per_sm, staged=False):
    """The `config` object of the bench line for a throughput-family case."""
    return {"workload": case["name"], "fluid_nodes": fluid_updates(case), "box_nodes": case["geometry"].n_nodes,
            "capsules": len(case["capsules"]), "markers": sum(len(c["verts"]) for c in case["capsules"]),
            "storage": storage, "l2": "inputs larger than L2 (distributions ~1 GB)",
            "parallelism": "replicas" if world > 1 else "1 GPU",
            "launch": {"threads": threads, "blocks_per_sm": blocks_per_sm,
                       "lattice_kernel": "staged (bulk copies)" if staged else "register gathers"}}


def reference_arm(args, rank):
    """--impl reference: the FP64 oracle, as it stands, on the host cores: one
    independent copy per core (one numpy thread each), each stepping a bounded
    x-slab sample of the workload (its own capsules, inlet and a pressure face
    at the cut) for the warm-up and timed steps."""
    from paper_2207_06043_gb300 import workloads as W
    if rank != 0:
        return
    case = W.throughput_case(**WORKLOADS[args.workload])
    sample = cpu_sample_case(case, REF_SAMPLE_X)
    sample["geometry"].sdf = None
    nproc = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        procs = max(1, min(nproc, int(avail // 1.5e9)))
    except (ValueError, OSError):
        procs = nproc
    if args.warmup:
        oracle_throughput(sample, 1, procs)       # untimed: spawn, imports, first step
    mlups, wall, nf = oracle_throughput(sample, args.steps, procs)
    samp = (f"x-slab [0,{REF_SAMPLE_X}) of the workload ({nf} fluid nodes, {len(sample['capsules'])} capsules), "
            f"{args.steps} steps, one copy per core on {procs} cores")
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(case, args.storage, args.gpus, args.threads, args.blocks_per_sm),
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": samp},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_survey(args):
    """--cpu-survey: the FP64 oracle on the host cores over the standard
    configurations, single-threaded and one independent copy per core at
    once (throughput): the small bifurcation in full (500 steps), windows of
    the deformable-capsule, batched-sweep (member 0), adjoint and throughput
    (its x-slab [0, 64) with 21 capsules) configurations.  No GPU is used."""
    from paper_2207_06043_gb300 import workloads as W
    nproc = os.cpu_count() or 1
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = None
    plan = [("small bifurcation 96x32x32, rigid sphere (full run)", W.bifurcation_small(), 500, 1.0e8),
            ("deformable capsule 256x96x64", W.deformable_capsule(), args.survey_window, 2.0e9),
            ("batched sweep member 0", W.sweep_member(0), args.survey_window, 2.0e9),
            ("adjoint 192x64x48 with capsule", W.adjoint_case(), args.survey_window, 1.0e9),
            ("throughput x-slab [0,64), 21 capsules", cpu_sample_case(W.throughput_case()), 3, 2.0e9)]
    out = {"nproc": nproc, "cpu_model": cpu_model(), "runs": []}
    for name, case, steps, mem in plan:
        case["geometry"].sdf = None
        m1, w1, nf = oracle_throughput(case, steps, 1)
        procs = nproc if avail is None else max(1, min(nproc, int(avail // mem)))
        mn, wn, _ = oracle_throughput(case, steps, procs)
        out["runs"].append({"config": name, "fluid_nodes": nf, "steps": steps, "single_thread_mlups": m1,
                            "single_thread_s": w1, "all_cores_mlups": mn, "all_cores_procs": procs,
                            "all_cores_s": wn})
        print(json.dumps({"progress": out["runs"][-1]}), file=sys.stderr, flush=True)
    print(json.dumps({"cpu_survey": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="throughput", choices=sorted(WORKLOADS) + ["sweep", "deformable"])
    ap.add_argument("--traj-out", default=None, help="deformable campaign: write the trajectories here (JSON)")
    ap.add_argument("--members", type=int, default=64, help="lattices of the batched sweep workload")
    ap.add_argument("--cpu-steps", type=int, default=1)
    ap.add_argument("--cpu-survey", action="store_true", help="time the oracle on the host over the configurations")
    ap.add_argument("--survey-window", type=int, default=50, help="steps of the survey's windows")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-parity", action="store_true", help="skip the oracle-parity leg")
    ap.add_argument("--no-sweep", action="store_true", help="skip the batched-sweep side measurement")
    ap.add_argument("--no-slabs", action="store_true", help="skip the slab-decomposition side measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the 16-bit storage side measurements")
    ap.add_argument("--sweep-members", type=int, default=64)
    ap.add_argument("--sweep-steps", type=int, default=100)
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--adjoint-ckpt", type=int, default=100)
    ap.add_argument("--threads", type=int, default=128)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--staged", action="store_true",
                    help="step the lattice with the staged (bulk-copy) kernel instead of the register-gather one")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if args.cpu_survey:
        if rank == 0:
            cpu_survey(args)
        return
    if args.workload == "sweep":
        sweep_bench(args, rank, world, local)
        return
    if args.workload == "deformable":
        if rank == 0:
            deformable_campaign(args, local)
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
    s.set_lattice_path(args.staged)
    s.step(args.warmup)

    # timed region, twice: in timing mode (CUDA events between the phases,
    # which then run one after another on the library's stream) and as graph
    # replays (the production schedule); nvidia-smi samples both
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    with ClockSampler(local) as clk:
        s.enable_timing(True)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        s.step(args.steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        kt = s.kernel_times()
        s.enable_timing(False)
        s.step(1)                       # re-enter graph mode (captures outside the timed region)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev[2].record(stream)
        s.step(args.steps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = ev[0].elapsed_time(ev[1])
    ms_graph = ev[2].elapsed_time(ev[3])
    ms_best = max_over_ranks(min(ms, ms_graph), dist, "cuda")
    value = whole_job_mlups(nf, args.steps, ms_best, world)
    launches = s.kernels_per_step() * args.steps

    bpu = BYTES_PER_UPDATE[args.storage]
    peak, peak_kind = load_peaks()
    lbm_ms = kt["lattice"] / args.steps
    achieved = bpu * nf / (lbm_ms * 1e-3) / 1e9
    # the captured traffic belongs to the register-gather kernel
    traffic = None if args.staged else lbm_traffic(args.workload, args.storage)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum, mean of two launches, "
                               f"lattice sources {lbm_source_hash()}" if traffic else
                               f"not captured for the lattice sources {lbm_source_hash()}"),
            "kernel": ("k_lbm_tile (staged by bulk copies)" if args.staged else "k_lbm") +
                      " (fused collide+stream, AA pattern)",
            "peak_source": f"{peak_kind} hbm_gbs", "ms_per_launch": lbm_ms,
            "algorithmic_bytes_per_launch": bpu * nf}
    s.close()

    step_bytes = bpu * nf
    out = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_best / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
           "config": workload_config(case, args.storage, world, args.threads, args.blocks_per_sm, args.staged),
           "roofline": roof,
           "step_roofline": {"bound": "hbm", "algorithmic_bytes_per_step": step_bytes,
                             "achieved": step_bytes / (ms_best / args.steps * 1e-3) / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": step_bytes / (ms_best / args.steps * 1e-3) / 1e9 / peak,
                             "note": "lattice bytes only (152 B per fluid node) over the whole step"},
           "kernel_ms_per_step": {k: v / args.steps for k, v in kt.items()},
           "ms_per_step_timed_events": ms / args.steps, "ms_per_step_graph": ms_graph / args.steps,
           "clocks": clk.summary(),
           "gpu_launches": launches}

    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_run(case, args)
    if rank == 0 and not args.no_parity:
        out["oracle_parity"] = oracle_parity()
    if rank == 0 and not args.no_adjoint:
        out["adjoint"] = adjoint_measure(args, case)
    if rank == 0 and not args.no_variants and args.storage == "f32":
        out["storage_variants"] = storage_variants(case, nf, staged=args.staged)
    if rank == 0 and not args.no_sweep:
        out["sweep"] = sweep_measure(args.sweep_members, args.sweep_steps, local, dist)
    if rank == 0 and not args.no_slabs:
        out["slabs"] = slab_measure(case, nf, out["ms_per_step"])
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(case, args.cpu_steps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def oracle_parity(steps=PARITY_STEPS):
    """Error of the CUDA path against the FP64 oracle on the small bifurcation
    (96x32x32, rigid sphere d = 12, 642 v) after `steps` steps, for each
    storage: velocity relative L2 over the fluid nodes and the largest
    centroid difference (lattice units)."""
    from paper_2207_06043_gb300 import workloads as W
    from oracle import lattice as L
    from oracle import sim
    c = W.bifurcation_small()
    g = c["geometry"]
    lat = L.Lattice(g.nx, g.ny, g.nz, c["tau"], g.tag, g.links, g.faces, g.periodic)
    o = sim.Simulation(lat, u_max=c["u_max"])
    for cap in c["capsules"]:
        o.add_body(cap["verts"], cap["tris"], cap["params"], cap.get("vel0"))
    t0 = time.perf_counter()
    o.step(steps)
    t_or = time.perf_counter() - t0
    _, uo = lat.macroscopic(o.f)
    fl = lat.fluid
    cen_o = o.stats(0)["centroid"]
    out = {"workload": c["name"].replace("500 steps", f"{steps} steps"), "steps": steps,
           "oracle_seconds": t_or}
    for st in ("f32", "f16", "bf16"):
        s = W.make_solver(c, storage=st)
        s.step(steps)
        _, u = s.read_fields()
        cen = s.read_capsule(0)["centroid"]
        s.close()
        out[st] = {"velocity_rel_l2": float(np.linalg.norm(u[fl] - uo[fl]) / np.linalg.norm(uo[fl])),
                   "centroid_max_abs": float(np.abs(cen - cen_o).max())}
    return out


def slab_measure(case, nf, ms_whole, n_slabs=4, steps=50):
    """The same workload stepped as x-slabs of one context on this GPU (the
    decomposition a multi-GPU run uses, with its halo copies and the capsules'
    whole-lattice member): whole-step MLUPS against the undivided context, and
    the bytes the ghost-plane copies move per step (what each cut sends to its
    neighbours on several GPUs)."""
    import torch
    from paper_2207_06043_gb300 import binding as B
    from paper_2207_06043_gb300 import workloads as W
    whole = W.make_solver(case)
    grp = B.slab_group(whole, n_slabs)
    whole.close()
    grp.step(5)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    grp.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    g = case["geometry"]
    ghost_planes = sum(lo + hi for _, _, lo, hi in grp.slabs)
    ny_p = g.ny + (0 if g.periodic[1] else 2)
    nz_p = g.nz + (0 if g.periodic[2] else 2)
    halo_bytes = ghost_planes * ny_p * nz_p * 19 * 4 * 2   # every slot of every padded node, read + written
    grp.close()
    return {"slabs": n_slabs, "plan": [list(x) for x in grp.slabs], "value": nf / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "ms_per_step": ms, "steps": steps, "overhead_vs_whole": ms / ms_whole - 1.0,
            "halo_bytes_per_step": int(halo_bytes),
            "note": "one GPU; each ghost plane copied from its owner after every step (all 19 slots of every node)"}


def sweep_measure(n_members, steps, local, dist):
    """The batched sweep as a side measurement of the default run: the sweep
    members stepped as one context (graph replay, autotuned launch shape)."""
    members = sweep_members(n_members)
    return sweep_run(members, steps, max(3, steps // 10), local, dist)


def storage_variants(case, nf, steps=100, staged=False):
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
        s.set_lattice_path(staged)
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


def _adjoint_run(c, n, Ks, lo, hi):
    """Time n plain forward steps, then one ibl_adjoint call of n steps per
    checkpoint interval K in Ks, on the lattice of case c (no capsules), each
    on its own context.  Each adjoint is timed on its second call (the first
    allocates its buffers and captures its graphs)."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    fwd = W.make_solver(c)
    fwd.step(10)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    e[0].record(stream)
    fwd.step(n)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms_f = e[0].elapsed_time(e[1])
    fwd.close()
    nf = fluid_updates(c)
    out = {"fluid_nodes": nf, "steps": n, "ms_forward": ms_f}
    for K in Ks:
        adj = W.make_solver(c)
        adj.step(10)
        adj.adjoint_flow(n, lo, hi, (1.0, 0.0, 0.0), ckpt_every=K)     # allocates the buffers, captures the graphs
        torch.cuda.synchronize()
        e[0].record(stream)
        J, gs, gr = adj.adjoint_flow(n, lo, hi, (1.0, 0.0, 0.0), ckpt_every=K)
        e[1].record(stream)
        torch.cuda.synchronize()
        ms_a = e[0].elapsed_time(e[1])
        adj.close()
        out[f"K{K}"] = {"ckpt_every": K, "segments": -(-n // K), "recomputed_steps": n - min(K, n),
                        "ms_adjoint_call": ms_a, "cost_vs_forward": ms_a / ms_f,
                        "mlups_adjoint": nf * n / (ms_a * 1e-3) / 1e6,
                        "J": J, "dJ_du_max": gs / c["u_max"], "dJ_dr_j": gr}
    return out


def _adjoint_capsule_run(c, n, Ks, w=(1.0, 0.5)):
    """Time n plain forward steps, then one capsule adjoint call (ibl_adjoint)
    of n steps per checkpoint interval K in Ks, on case c (one soft capsule),
    each on its own context; each adjoint is timed on its second call."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    fwd = W.make_solver(c)
    fwd.step(10)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    e[0].record(stream)
    fwd.step(n)
    e[1].record(stream)
    torch.cuda.synchronize()
    ms_f = e[0].elapsed_time(e[1])
    fwd.close()
    nf = fluid_updates(c)
    out = {"fluid_nodes": nf, "steps": n, "ms_forward": ms_f, "objective": f"{w[0]} D + {w[1]} offset"}
    for K in Ks:
        adj = W.make_solver(c)
        adj.step(10)
        state = adj.save_state()
        adj.adjoint(n, w, ckpt_every=K)          # allocates the buffers, captures the graphs
        adj.load_state(state)
        torch.cuda.synchronize()
        e[0].record(stream)
        g = adj.adjoint(n, w, ckpt_every=K)
        e[1].record(stream)
        torch.cuda.synchronize()
        ms_a = e[0].elapsed_time(e[1])
        adj.close()
        out[f"K{K}"] = {"ckpt_every": K, "segments": -(-n // K), "recomputed_steps": n - min(K, n),
                        "ms_adjoint_call": ms_a, "cost_vs_forward": ms_a / ms_f,
                        "dJ_dCa": g[0], "dJ_du_max": g[1], "dJ_dr_j": g[2]}
    return out


def adjoint_measure(args, case):
    """The discrete adjoint against the same number of plain forward steps:
      (a) the adjoint workload as specified (192x64x48 bifurcation, junction
          radius 4 lu, one soft capsule d = 27 of 2562 vertices, Ca = 0.01,
          2000 steps), the capsule objective D + 0.5 offset (ibl_adjoint) with
          checkpoints every --adjoint-ckpt steps (default 100: each earlier
          segment is recomputed from its checkpoint while its tape is
          rebuilt) and with one segment (whole tape in HBM);
      (b) the throughput workload's lattice without capsules (12.6 M nodes,
          100 steps, one segment), the flow objective (ibl_adjoint_flow),
          whose HBM fraction is reported at 336 B per node and step."""
    from paper_2207_06043_gb300 import workloads as W
    out = {"note": "each timed call runs the forward sweep (checkpoints, or the tape of the only segment), "
                   "the recompute of every earlier segment with its tape, and the reverse sweep; buffers and "
                   "graphs come from a first, untimed call"}
    ca = W.adjoint_case()
    Ks = [args.adjoint_ckpt] + ([args.adjoint_steps] if args.adjoint_ckpt < args.adjoint_steps else [])
    r = _adjoint_capsule_run(ca, args.adjoint_steps, Ks)
    r["cost_vs_forward"] = r[f"K{args.adjoint_ckpt}"]["cost_vs_forward"]
    out["adjoint_workload"] = dict(r, workload="bifurcation 192x64x48, D 36, 45 deg, junction radius 4 lu, "
                                               "capsule d=27 (2562 v), Ca 0.01")
    ct = dict(case, capsules=[])
    g = ct["geometry"]
    r = _adjoint_run(ct, 100, [100], (4, int(g.info["yc"]), 0), (52, g.ny, g.nz))
    bpu = 168 + 168            # forward step writing the tape, adjoint step (B per fluid node and step)
    peak, kind = load_peaks()
    ach = bpu * r["fluid_nodes"] * r["steps"] / (r["K100"]["ms_adjoint_call"] * 1e-3) / 1e9
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


def sweep_members(n):
    """The sweep's members, generated in spawned worker processes."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_sweep_member, range(n))


def sweep_run(members, steps, warmup, local, dist):
    """Step the members together as one context (one launch per kernel per
    step for all lattices, CUDA graphs), launch shape chosen by the library's
    autotuner.  MLUPS counts the fluid nodes of the members still running (a
    capsule that breaks stops its lattice, as the damage rule says)."""
    import torch
    from paper_2207_06043_gb300 import binding
    from paper_2207_06043_gb300 import workloads as W
    nf = [fluid_updates(c) for c in members]
    ens = binding.ensemble([W.make_solver(c) for c in members])
    ens.step(warmup, allow_damage=True)
    thr, bps, _ = ens.autotune(4)
    n_m = len(members)

    def steps_done():
        return [ens.member_steps(m) for m in range(n_m)]

    stream = torch.cuda.current_stream()
    # lattice-kernel time per step from a timing-mode pass
    ens.enable_timing(True)
    c0 = steps_done()
    ens.step(steps, allow_damage=True)
    c1 = steps_done()
    kt = ens.kernel_times()
    ens.enable_timing(False)
    ens.step(1, allow_damage=True)       # back to graph replay (captures outside the timed region)
    c1 = steps_done()
    upd_timing = sum(nf[m] * (c1[m] - c0[m] - 1) for m in range(n_m))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        ens.step(steps, allow_damage=True)
        e1.record(stream)
        torch.cuda.synchronize()
    c2 = steps_done()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    world = dist.get_world_size() if dist else 1
    upd = sum(nf[m] * (c2[m] - c1[m]) for m in range(n_m))
    bpu = BYTES_PER_UPDATE["f32"]
    peak, peak_kind = load_peaks()
    achieved = bpu * upd_timing / (kt["lattice"] * 1e-3) / 1e9 if kt["lattice"] > 0 else 0.0
    stopped = [m for m in range(n_m) if c2[m] - c1[m] < steps]
    out = {"value": world * upd / (ms * 1e-3) / 1e6, "unit": "MLUPS", "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps,
           "workload": f"batched sweep: {n_m} bifurcations of uneven size, one capsule each",
           "fluid_nodes": int(sum(nf)), "box_nodes": int(sum(c["geometry"].n_nodes for c in members)),
           "running_members": n_m - len(stopped),
           "stopped_members": [{"member": m, "Ca": members[m]["capsules"][0]["params"]["Ca"],
                                "steps_done": c2[m]} for m in stopped],
           "launch": {"threads": thr, "blocks_per_sm": bps, "chosen_by": "ibl_autotune"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "k_lbm (all members in one launch)", "peak_source": f"{peak_kind} hbm_gbs"},
           "kernel_ms_per_step": {k: v / steps for k, v in kt.items()},
           "clocks": clk.summary(), "gpu_launches": ens.kernels_per_step() * steps}
    ens.close()
    return out


def sweep_bench(args, rank, world, local):
    """--workload sweep: the batched sweep as the bench's own workload."""
    members = sweep_members(args.members)
    import torch
    torch.cuda.set_device(local)
    torch.zeros(1, device="cuda")
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    r = sweep_run(members, args.steps, args.warmup, local, dist)
    out = {"metric": METRIC, "value": r["value"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": r["workload"], "fluid_nodes": r["fluid_nodes"], "box_nodes": r["box_nodes"],
                      "running_members": r["running_members"], "l2": "inputs larger than L2",
                      "launch": r["launch"]},
           "roofline": r["roofline"], "kernel_ms_per_step": r["kernel_ms_per_step"],
           "stopped_members": r["stopped_members"], "clocks": r["clocks"], "gpu_launches": r["gpu_launches"]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def deformable_campaign(args, local):
    """--workload deformable: the deformable-capsule configuration in full:
    half-angles 30, 45 and 60 deg x Ca 0.005, 0.01 and 0.05 (256x96x64 duct,
    D = 48, junction rounding 8 lu, capsule d = 36 of 2562 vertices, Re = 10),
    each stored as FP32, FP16 and BF16 (FP32 arithmetic), --steps steps
    (default 20000 here) with the capsule's FP64 diagnostics read every 100
    steps.  Prints one JSON line: MLUPS over all runs and, per run, the final
    centroid, branch offset, Taylor D (final and largest), the largest volume
    drift, and for the 16-bit forms the largest centroid and D deviation from
    the FP32 run over the trajectory."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    torch.cuda.set_device(local)
    torch.zeros(1, device="cuda")
    steps = args.steps
    every = 100
    runs = []
    traj_all = {}
    total_upd, total_ms = 0, 0.0
    stream = torch.cuda.current_stream()
    for th in (30.0, 45.0, 60.0):
        for Ca in (0.005, 0.01, 0.05):
            case = W.deformable_capsule(th, Ca)
            nf = fluid_updates(case)
            yc = case["geometry"].info["yc"]
            per_storage = {}
            for st in ("f32", "f16", "bf16"):
                s = W.make_solver(case, storage=st)
                s.step(0)
                V0 = s.read_capsules(1)[0]["volume"]
                traj = []
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                done_total = 0
                torch.cuda.synchronize()
                e0.record(stream)
                for _ in range(steps // every):
                    done, _ = s.step(every, allow_damage=True)
                    done_total += done
                    c = s.read_capsules(1)[0]
                    traj.append((done_total, *c["centroid"].tolist(), c["volume"], c["taylor_D"], c["dS"],
                                 c["max_stretch"]))
                    if done < every:
                        break
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                s.close()
                total_upd += nf * done_total
                total_ms += ms
                per_storage[st] = np.array(traj)
            t32 = per_storage["f32"]
            rec = {"half_angle": th, "Ca": Ca, "fluid_nodes": nf}
            for st, t in per_storage.items():
                last = t[-1]
                r = {"steps_done": int(last[0]), "centroid": [round(v, 6) for v in last[1:4]],
                     "branch_offset": round(last[2] - yc, 6), "taylor_D_final": round(last[5], 6),
                     "taylor_D_max": round(float(t[:, 5].max()), 6),
                     "volume_drift_max": float(np.abs(t[:, 4] / V0 - 1.0).max()),
                     "dS_max": round(float(t[:, 6].max()), 6), "max_stretch_max": round(float(t[:, 7].max()), 6)}
                if st != "f32":
                    n = min(len(t), len(t32))
                    r["centroid_dev_vs_f32_max"] = float(np.abs(t[:n, 1:4] - t32[:n, 1:4]).max())
                    r["taylor_D_dev_vs_f32_max"] = float(np.abs(t[:n, 5] - t32[:n, 5]).max())
                rec[st] = r
                traj_all[f"th{th:g}_Ca{Ca:g}_{st}"] = t.tolist()
            runs.append(rec)
            print(json.dumps({"progress": rec}), file=sys.stderr, flush=True)
    if args.traj_out:
        with open(args.traj_out, "w") as fh:
            json.dump({"columns": ["step", "cx", "cy", "cz", "volume", "taylor_D", "dS", "max_stretch"],
                       "runs": traj_all}, fh)
    out = {"metric": METRIC, "value": total_upd / (total_ms * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
           "steps": steps, "warmup": 0, "ms_per_step": total_ms / (len(runs) * 3 * steps),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f16/bf16 storage",
           "data": "synthetic",
           "config": {"workload": "deformable capsule 256x96x64, D 48, junction rounding 8 lu, d 36 (2562 v), "
                                  "Re 10; half-angle x Ca x storage campaign", "stats_every": every,
                      "note": "value and ms_per_step include the FP64 diagnostics read every 100 steps"},
           "runs": runs}
    print(json.dumps(out), flush=True)


def e2e_run(case, args, chunk=10):
    """The same metric through the public API from host buffers.  Set-up: the
    context is created from the host arrays (every input copied host ->
    device, topology and work lists built, initial state written).  Then the
    time steps in chunks of `chunk`, each chunk followed by a device -> host
    read of every capsule's FP64 diagnostics (ibl_read_capsules: centroid,
    volume, area, Taylor D, stretch, velocity), and a read of the fields to
    the host at the end.  `value` covers both; `steady` covers the
    stepping with its per-chunk reads alone."""
    import torch
    from paper_2207_06043_gb300 import workloads as W
    g = case["geometry"]
    nf = fluid_updates(case)
    h2d = g.tag.nbytes + g.links.nbytes + sum(f.velocity.nbytes for f in g.faces if f.velocity is not None)
    h2d += sum(c["verts"].nbytes + c["tris"].nbytes for c in case["capsules"])
    # the caller's result buffers: page-locked host memory, allocated once
    rho_h = torch.empty(g.n_nodes, dtype=torch.float32, pin_memory=True)
    u_h = torch.empty((g.n_nodes, 3), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = W.make_solver(case, storage=args.storage)
    s.set_launch(args.threads, args.blocks_per_sm)
    s.set_lattice_path(args.staged)
    s.step(0)                               # set-up: uploads, work lists, initial state
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    d2h = 0
    left = args.steps
    while left > 0:
        k = min(chunk, left)
        s.step(k)
        left -= k
        if case["capsules"]:
            s.read_capsules(len(case["capsules"]))
            d2h += 18 * 8 * len(case["capsules"])
    rho, u = s.read_fields(out=(rho_h, u_h))
    d2h += rho.numel() * rho.element_size() + u.numel() * u.element_size()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    s.close()
    return {"value": nf * args.steps / (t2 - t0) / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": h2d / args.steps,
            "d2h_bytes_per_step": d2h / args.steps, "setup_ms": 1e3 * (t1 - t0),
            "steady": {"value": nf * args.steps / (t2 - t1) / 1e6, "unit": "MLUPS",
                       "ms_per_step": 1e3 * (t2 - t1) / args.steps, "chunk": chunk,
                       "d2h_bytes_per_step": d2h / args.steps},
            "note": f"value includes the set-up from host arrays (setup_ms); steady = the steps with a read of "
                    f"every capsule's diagnostics after each chunk of {chunk} steps and the fields at the end "
                    f"(into page-locked host buffers)"}


if __name__ == "__main__":
    main()
