#!/usr/bin/env python
"""Throughput benchmark of the reactive-mixture LBM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp64|fp32|fp32c64|fp16] [--variants LIST]
                    [--impl ours|reference]

One step = one pass of the whole hot path over the workload: pull streaming,
boundary reconstruction, moments, temperature Newton, relaxation, gradients,
diffusion velocities, reaction sub-steps and collision of all M+1 lattices.
Metric: node-updates/s = fluid-node steps/s x (M+2) (every fluid node
advances M species + f + g per step, the slaved species included), i.e.
MLUPS x 11.  Solid nodes (the microtube's staircase wall) are not updated
and not counted.

Default workload: the 600x40x40 D3Q27 microtube (960 000 nodes, 674 400
fluid), the largest configuration of the method's workloads that fits one
GPU, in FP64 (the paper's precision).  The mixed-precision storage paths of
the same workload, and on the tube the same tube with off-grid TMS targets
(in the headline's precision), are timed in the same run and reported under
"variants".

Timing: W untimed steps, then K steps each bracketed by CUDA events on the
library's stream (torch's current stream); when the populations fit in L2
(129 MB), a 256 MB buffer is overwritten between timed steps, outside the
events.  Per-kernel-group device times come from a second pass of K steps
with events the library records around each launch group
(lbm_step_timed).  Under torchrun every rank advances its own independent,
seeded copy of the workload (weak scaling, no collective on the data path);
rank 0 prints the max-over-ranks time.

Roofline: HBM bandwidth over the whole step (algorithmic population bytes
2 L Q s per fluid node, read and write once, divided by the device time of
the step) against MEASURED_PEAKS.json's copy bandwidth; beside it the ALU
roof: executed FP64 (or FP32) FLOP per fluid node from the committed ncu
counters (profiles/step_counters.txt) over the step time, against the FMA
throughput measured in this run (lbm_fma_peak).

--impl reference times the CPU oracle (plain FP64 numpy) as it stands on a
bounded sample of the workload (the microtube: a 20x40x40 segment with the
same wall, inlet and outlet), K steps after W warm-up steps, one process,
on rank 0 only.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")     # each oracle process runs on one host thread

L2_BYTES = 129 * 1024 * 1024
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

WORKLOADS = {"reactor": "homogeneous reactor 16^3 periodic D3Q27, M=9, 21 reactions, "
                        "phi=0.5, 1200 K (+1e-3 seeded perturbation), 1 atm",
             "flame": "quasi-1D premixed flame 1024x4x4 D3Q27, inlet/outlet, M=9, "
                      "21 reactions, phi=0.5, tanh ignition kernel at x=256",
             "channel": "2D microchannel 2000x40 D2Q9, TMS walls 300->1500 K ramp, parabolic "
                        "inlet, LODI outlet, M=9, 21 reactions, phi=0.5",
             "tube": "3D microtube 600x40x40 D3Q27, circular staircase wall r=19 (TMS, "
                     "300->1500 K ramp), inlet 1 m/s, LODI outlet, M=9, 21 reactions, phi=0.5",
             "box": "perturbed periodic box 128x64x64 D3Q27, M=9, 21 reactions, "
                    "1400 K +-2%, |u| <= 1 m/s (profiling case larger than L2)"}

# storage / arithmetic modes: (library precision, chemistry in native FP64, dtype text)
MODES = {
    "fp64": ("fp64", 0, "f64"),
    "fp32": ("fp32", 0, "f32 storage and lattice arithmetic; temperature Newton and "
                        "chemistry in float-float (two FP32 words, ~48-bit significand)"),
    "fp32c64": ("fp32", 1, "f32 storage and lattice arithmetic; temperature Newton and "
                           "chemistry in native FP64"),
    "fp16": ("fp16", 0, "f16 offset storage, f32 lattice arithmetic; temperature Newton "
                        "and chemistry in float-float"),
}
DEFAULT_VARIANTS = "fp32,fp32c64,fp16,offgrid"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=150)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="tube", choices=sorted(WORKLOADS))
    p.add_argument("--precision", default="fp64", choices=sorted(MODES),
                   help="storage / arithmetic of the headline line")
    p.add_argument("--variants", default=DEFAULT_VARIANTS,
                   help="comma list of further modes timed on the same workload "
                        "('none' for none)")
    p.add_argument("--chem-lanes", type=int, default=0, choices=[0, 1, 4, 8],
                   help="chemistry placement (0: the library default)")
    p.add_argument("--collide-split", type=int, default=-1, choices=[-1, 0, 1],
                   help="collision placement (-1: the library default)")
    p.add_argument("--autotune", action="store_true",
                   help="let the library's autotuner choose the placement before timing")
    p.add_argument("--substeps", type=int, default=0,
                   help="reaction sub-steps l (Eq. R3); 0 keeps the workload's value")
    p.add_argument("--nx", type=int, default=0,
                   help="length of the flame, channel or tube (0: the workload's own)")
    p.add_argument("--serve-scale", type=float, default=0.02,
                   help="step scale of the serving mix timed beside the headline (0: skip)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def _workload(name, seed, nx=0):
    from lbm_workloads import fields
    kw = {"nx": nx} if nx else {}
    return {"reactor": lambda: fields.reactor(seed=seed),
            "flame": lambda: fields.flame_1d(seed=seed, **kw),
            "channel": lambda: fields.channel_2d(seed=seed, **kw),
            "tube": lambda: fields.microtube(seed=seed, **kw),
            "box": lambda: fields.perturbed_box((128, 64, 64), "D3Q27", seed=seed,
                                                dx=12.5e-6, amp_u=1.0)}[name]()


# bounded samples of each workload for the oracle (CPU) timings: the same
# geometry, boundaries and fields on a shorter domain
ORACLE_SAMPLES = {"tube": ("tube", 20, "20x40x40 segment of the microtube (same wall, inlet, "
                                       "outlet and fields)"),
                  "flame": ("flame", 64, "64x4x4 flame (same inlet, outlet and fields)"),
                  "channel": ("channel", 100, "100x40 channel (same walls, inlet, outlet)"),
                  "reactor": ("reactor", 0, "the full 16^3 reactor"),
                  "box": ("box", 0, "the full 128x64x64 box")}


def fluid_nodes(w):
    n = int(w["P"].size)
    if w.get("solid") is not None:
        n -= int(w["solid"].sum())
    return n


def boundary_spec(w):
    """Boundary description of a workload (faces, inlet, outlet, walls,
    solid nodes), or None for a periodic box."""
    keys = ("faces", "inlet", "outlet", "wall_T", "solid", "solid_kind", "wall_dist",
            "wall_normal")
    if all(f == "periodic" for f in w.get("faces", ("periodic",) * 6)) and w.get("solid") is None:
        return None
    return {k: w[k] for k in keys if k in w}


def max_over_ranks(x, pg):
    """The largest x over all ranks (x itself without a process group)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t[0])


def node_updates_per_s(nodes_per_rank, steps, world, species, seconds):
    """Whole-job throughput: every rank advances its own copy of the
    workload (weak scaling); a node update is one lattice of one fluid node,
    M + 2 per node-step."""
    return nodes_per_rank * steps * world * (species + 2) / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling every 100 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def launch_groups(launch, has_bnd):
    """Names of the two timed launch groups of a step (lbm_step_timed): the
    kernels before the collision, and the collision."""
    g0 = (["k_boundary", "k_chem"] if has_bnd else []) + \
        ["k_mchem" if launch["chem_lanes"] > 1 else "k_moments"]
    return ["+".join(g0), "k_prep+k_coll" if launch["collide_split"] else "k_collide"]


def launches_per_step(launch, has_bnd):
    """Kernels one step launches: the moments with the reaction sub-steps
    (k_moments or k_mchem), the collision (k_collide, or k_prep + k_coll);
    with interface nodes also the boundary kernel and the interface nodes'
    sub-steps (k_chem)."""
    return 1 + (2 if has_bnd else 0) + (2 if launch["collide_split"] else 1)


def step_counters(workload, mode):
    """Per-fluid-node counters of a whole step from the committed ncu
    summary (profiles/step_counters.txt): {"fp32_flop", "fp64_flop",
    "dram_bytes", "kernels"}, or None when it has no line for the pair."""
    path = os.path.join(ROOT, "profiles", "step_counters.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if tuple(f[:2]) == (workload, mode):
            return {"fp32_flop": float(f[2]), "fp64_flop": float(f[3]),
                    "dram_bytes": float(f[4]), "kernels": f[5] if len(f) > 5 else ""}
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def host_info():
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


# ---------------------------------------------------------------- oracle legs
def _oracle_sample(workload):
    name, nx, text = ORACLE_SAMPLES[workload]
    return _workload(name, 0, nx), text


def _oracle(w):
    from lbm_workloads.mechanism import h2_air_synthetic
    from oracle import OracleLBM, thermo
    mech = h2_air_synthetic()
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], T_max=w["T_max"],
                  substeps=w["substeps"], boundaries=boundary_spec(w))
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    return o, mech.n_species


def _oracle_worker(job):
    """One oracle process: `warm` untimed steps, then `steps` timed ones;
    returns (fluid node-updates, seconds)."""
    workload, warm, steps = job
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"
    w, _ = _oracle_sample(workload)
    o, M = _oracle(w)
    o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    return fluid_nodes(w) * steps * (M + 2), time.perf_counter() - t0


def run_reference(args, rank):
    """The CPU oracle as it stands on the bounded sample of the workload:
    W warm-up steps, then K timed steps, one process on one host thread."""
    if rank != 0:
        return
    w, text = _oracle_sample(args.workload)
    o, M = _oracle(w)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    Nf = fluid_nodes(w)
    v = Nf * args.steps * (M + 2) / dt
    line = {
        "impl": "reference", "metric": "node-updates/s", "value": v, "unit": "node-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample": text,
                   "nodes": int(w["P"].size), "fluid_nodes": Nf, "precision": "fp64",
                   "l2": "oracle on host cores"},
        "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps of the {text} after {args.warmup} "
                                   f"warm-up steps, numpy single-threaded",
                         **host_info()},
        "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(workload, budget_s=12.0):
    """The oracle on the host cores on a bounded sample of the workload: one
    process (one thread), then one process per core, each advancing its own
    copy of the sample for the same number of steps (processes started with
    spawn; throughput = all node-updates / wall time)."""
    import multiprocessing as mp
    info = host_info()
    _, secs = _oracle_worker((workload, 1, 1))
    n = max(1, int(budget_s / max(secs, 1e-6)))
    u1, s1 = _oracle_worker((workload, 0, n))
    cores = max(1, info["nproc"] or 1)
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(workload, 0, n)] * cores)
    wall = time.perf_counter() - t0
    total = sum(u for u, _ in res)
    _, text = _oracle_sample(workload)
    return {"value": total / wall, "unit": "node-updates/s", "cores": cores, "kind": "oracle",
            "one_core": u1 / s1,
            "sample": f"{n} steps of the {text} per process; {cores} spawned processes "
                      f"(one numpy thread each; wall time includes their start-up), and "
                      f"one process alone for one_core",
            **info}


# ---------------------------------------------------------------- GPU legs
def make_solver(lbm, mech, w, mode, device):
    prec, chem64, _ = MODES[mode]
    kw = dict(boundary_spec(w) or {})
    s = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"], precision=prec,
                   substeps=w["substeps"], T_max=w["T_max"], device=device,
                   chem_fp64=chem64, **kw)
    s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    return s


def time_steps(solver, steps, stream, flush_buf):
    """Device milliseconds of `steps` single steps, each bracketed by events
    on the library stream (the L2 flush buffer, if any, is overwritten
    between them outside the events)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        if flush_buf is not None:
            flush_buf.zero_()
        starts[k].record(stream)
        solver.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    solver.synchronize()
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends))


def roofline(workload, mode, info, Nf, ms_per_step, peaks, fma):
    """HBM roof of the whole step and, beside it, the ALU roof of the
    executed operation counts (profiles/step_counters.txt)."""
    alg_bytes = 2 * info.L * info.Q * info.bytes_per_population       # per fluid node-step
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    achieved = alg_bytes * Nf / (ms_per_step * 1e-3) / 1e9
    cnt = step_counters(workload, mode)
    fp64 = mode == "fp64"
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": achieved / hbm_peak,
            "traffic": cnt["dram_bytes"] * Nf if cnt else None,
            "kernel": "whole step (all launches of one step)",
            "alg_bytes_per_node": alg_bytes,
            "peak_source": ("MEASURED_PEAKS.json hbm_gbs (measured copy)" if "hbm_gbs" in peaks
                            else "fallback 6.8 TB/s")}
    if cnt:
        key = "fp64_flop" if fp64 else "fp32_flop"
        peak = fma["fp64" if fp64 else "fp32"]
        tf = cnt[key] * Nf / (ms_per_step * 1e-3) / 1e12
        roof["alu"] = {"bound": "alu", "pipe": "fp64" if fp64 else "fp32",
                       "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                       "frac": tf / peak if peak else None,
                       "flop_per_node": cnt[key],
                       "flop_kind": "executed (ncu: add + mul + 2 fma thread instructions)",
                       "peak_source": "lbm_fma_peak measured in this run (FMA chains)"}
    return roof


def served_mix(mech, step_scale, device):
    """The serving mix (64 seeded requests, Poisson arrivals with mean 50 ms,
    reactor / flame / channel solves of 4k to 262k nodes) with every
    request's 1k-10k steps scaled by step_scale: the continuous-batching
    server in FP32 storage (least remaining work first) and, as the
    baseline, the plain FP64 path one request at a time.  Time-to-result =
    completion minus arrival on the host clock."""
    from lbm_workloads.fields import serving_mix
    from paper_2108_07605_gb300 import serve

    def stream():
        st = serving_mix(seed=0, mech=mech)
        for _, w in st:
            w["steps"] = max(1, int(round(w["steps"] * step_scale)))
        return st
    budget = int(40e9)
    srv = serve.Server(mech, budget, chunk=100, precision="fp32", device=device)
    done = srv.run(stream())
    ours = serve.summarize(done, srv.elapsed, srv.node_updates)
    base = serve.run_serial(mech, stream(), budget, "fp64", device=device)
    keys = ("p50_time_to_result_s", "p99_time_to_result_s", "node_updates_per_s",
            "makespan_s", "requests")
    return {"mix": f"64 seeded requests (Poisson arrivals, mean 50 ms; reactor, flame and "
                   f"channel solves of 4k-262k nodes), the stated 1k-10k steps scaled by "
                   f"{step_scale}",
            "batched_fp32_srpt": {k: ours[k] for k in keys},
            "serial_fp64": {k: base[k] for k in keys},
            "failed": len(ours["failed"]) + len(base["failed"]),
            "throughput_vs_serial_fp64": ours["node_updates_per_s"] / base["node_updates_per_s"],
            "p99_vs_serial_fp64": ours["p99_time_to_result_s"] / base["p99_time_to_result_s"],
            "p50_vs_serial_fp64": ours["p50_time_to_result_s"] / base["p50_time_to_result_s"]}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_2108_07605_gb300 import lbm
    from lbm_workloads.mechanism import h2_air_synthetic

    mech = h2_air_synthetic()
    w = _workload(args.workload, seed=rank, nx=args.nx)
    if args.substeps:
        w["substeps"] = args.substeps
    N = int(w["P"].size)
    Nf = fluid_nodes(w)
    M = mech.n_species
    has_bnd = boundary_spec(w) is not None
    peaks = measured_peaks()
    fma = {"fp64": lbm.lbm_fma_peak(True), "fp32": lbm.lbm_fma_peak(False)}
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_for(info):
        """The flush buffer when the state fits in L2, else None."""
        return flush_buf if 2 * info.L * info.Q * N * info.bytes_per_population < 2 * L2_BYTES \
            else None

    solver = make_solver(lbm, mech, w, args.precision, local)
    info = solver.info
    flush = flush_for(info)
    solver.step(args.warmup)
    solver.synchronize()
    # kernel placement: the library's default for this grid and precision,
    # the values given on the command line, or --autotune (trial steps on the
    # current state; the solve itself is not advanced)
    if args.autotune:
        launch = solver.autotune(trial_steps=3)
    else:
        solver.set_launch(args.chem_lanes or -1, args.collide_split)
        launch = solver.launch()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        total_ms = time_steps(solver, args.steps, stream, flush)
    # per-group device times: a second pass of the same number of steps with
    # events around every launch group (lbm_step_timed), L2 flushed likewise,
    # from the initial state again (a workload's stated step count, such as
    # the reactor's 200 through ignition, is not exceeded)
    solver.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    solver.step(args.warmup)
    kms = [0.0, 0.0]
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        kms = lbm.lbm_step_timed(solver.h, 1, kms)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, pg)
    if pg:
        pg.barrier()
    ms_per_step = total_ms / args.steps
    value = node_updates_per_s(Nf, args.steps, world, M, total_ms * 1e-3)
    roof = roofline(args.workload, args.precision, info, Nf, ms_per_step, peaks, fma)
    names = launch_groups(launch, has_bnd)

    # end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        host = {k: np.ascontiguousarray(w[k]).reshape(-1) for k in ("P", "u", "T", "Y")}
        pinned = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
        outs = {k: torch.empty(n, dtype=torch.float64).pin_memory()
                for k, n in (("rho", N), ("u", 3 * N), ("T", N), ("Y", M * N), ("E", N))}
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        t0 = time.perf_counter()
        lbm.lbm_init_fields_pressure(solver.h, pinned["P"], pinned["u"], pinned["T"],
                                     pinned["Y"])
        lbm.lbm_step(solver.h, args.steps)
        lbm.lbm_moments(solver.h, outs["rho"], outs["u"], outs["T"], outs["Y"], outs["E"])
        e2e_s = max_over_ranks(time.perf_counter() - t0, pg)
        h2d = sum(v.numel() * 8 for v in pinned.values())
        d2h = sum(v.numel() * 8 for v in outs.values())
        e2e = {"value": node_updates_per_s(Nf, args.steps, world, M, e2e_s),
               "unit": "node-updates/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "timed": "init from host fields + K steps + all fields read back to host"}
    solver.close()

    # the other storage / arithmetic modes on the same workload
    variants = {}
    for mode in [v for v in args.variants.split(",") if v and v != "none"]:
        if mode == "offgrid" and args.workload == "tube":
            # the same tube with off-grid TMS targets (wall distance and
            # inward normal per interface node, Sec. 4.2.2 last paragraph),
            # in the headline's precision
            from lbm_workloads import fields
            kw = {"nx": args.nx} if args.nx else {}
            wo = fields.microtube(seed=rank, offgrid=True, **kw)
            if args.substeps:
                wo["substeps"] = args.substeps
            s = make_solver(lbm, mech, wo, args.precision, local)
            s.step(args.warmup)
            s.synchronize()
            if pg:
                pg.barrier()
            vms = max_over_ranks(time_steps(s, args.steps, stream, flush_for(s.info)), pg)
            s.close()
            vval = node_updates_per_s(Nf, args.steps, world, M, vms * 1e-3)
            variants[mode] = {"value": vval, "unit": "node-updates/s",
                              "ms_per_step": vms / args.steps,
                              "dtype": MODES[args.precision][2] + ", off-grid TMS targets",
                              "speedup_vs_headline": vval / value,
                              "extra_ms_per_step": vms / args.steps - ms_per_step}
            continue
        if mode == args.precision or mode not in MODES:
            continue
        s = make_solver(lbm, mech, w, mode, local)
        s.step(args.warmup)
        s.synchronize()
        vinfo = s.info
        if pg:
            pg.barrier()
        vms = max_over_ranks(time_steps(s, args.steps, stream, flush_for(vinfo)), pg)
        vlaunch = s.launch()
        s.close()
        vms_step = vms / args.steps
        vval = node_updates_per_s(Nf, args.steps, world, M, vms * 1e-3)
        variants[mode] = {"value": vval, "unit": "node-updates/s", "ms_per_step": vms_step,
                          "dtype": MODES[mode][2], "speedup_vs_headline": vval / value,
                          "launch": vlaunch,
                          "roofline": roofline(args.workload, mode, vinfo, Nf, vms_step, peaks,
                                               fma)}

    served = served_mix(mech, args.serve_scale, local) if args.serve_scale > 0 else None

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args.workload)
    line = {
        "metric": "node-updates/s", "value": value, "unit": "node-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": MODES[args.precision][2], "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "nodes": N, "fluid_nodes": Nf,
                   "lattice": w["lattice"], "species": M, "precision": args.precision,
                   "substeps": w["substeps"],
                   "node_steps_per_s": Nf * args.steps * world / (total_ms * 1e-3),
                   "l2": "256 MB buffer overwritten between timed steps" if flush is not None
                   else "state larger than L2", "parallelism": f"replicas x{world}",
                   "launch": launch},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step(launch, has_bnd) * args.steps,
        "kernel_ms_per_step": {names[0]: kms[0] / args.steps, names[1]: kms[1] / args.steps},
        "fma_peak_tflops": fma,
        "variants": variants,
        "served": served,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
