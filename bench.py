#!/usr/bin/env python
"""Throughput benchmark of the reactive-mixture LBM step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                    [--precision fp32|fp64|fp16] [--impl ours|reference]

One step = one pass of the whole hot path over the workload: pull streaming,
boundary reconstruction, moments, temperature Newton, relaxation, gradients,
diffusion velocities, reaction sub-steps and collision of all M+1 lattices.
Metric: node-updates/s = lattice node-steps/s x (M+2) (every node advances
M species + f + g per step, the slaved species included), i.e. MLUPS x 11.

Timing: W untimed steps (with --autotune, then the library's autotuner:
trial steps that leave the solve untouched), then K steps each bracketed by
CUDA events on the
library's stream (torch's current stream); when the populations fit in L2
(129 MB), a 256 MB buffer is overwritten between timed steps, outside the
events.  Per-kernel device times come from a second pass of K steps with
events the library records around each launch group (lbm_step_timed).  Under torchrun every rank advances its
own independent, seeded copy of the workload (weak scaling, no collective on
the data path); rank 0 prints the max-over-ranks time.

--impl reference times the CPU oracle (plain FP64 numpy, one thread) on the
same workload, K steps after W warm-up steps, on rank 0 only.
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
    os.environ.setdefault(_v, "1")     # the oracle legs run on one host thread

L2_BYTES = 129 * 1024 * 1024
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
FP64_PEAK_TFLOPS = 1.25     # nominal FP64 rate of GB300 (152 SMs), per the pool's recipe
# FP32 rate from the unit counts and the clock: 152 SMs x 128 FP32 lanes x 2
# FLOP per FMA x 2.07 GHz (the maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="flame", choices=sorted(WORKLOADS))
    p.add_argument("--chem-lanes", type=int, default=0, choices=[0, 1, 4, 8],
                   help="chemistry placement (0: the library default)")
    p.add_argument("--collide-split", type=int, default=-1, choices=[-1, 0, 1],
                   help="collision placement (-1: the library default)")
    p.add_argument("--autotune", action="store_true",
                   help="let the library's autotuner choose the placement before timing")
    p.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16"],
                   help="population storage: fp64 (all FP64), fp32 (mixed: FP32 storage and "
                        "collision, float-float temperature and chemistry; the default), fp16 "
                        "(FP16 offsets, the fp32 path's arithmetic)")
    p.add_argument("--substeps", type=int, default=0,
                   help="reaction sub-steps l (Eq. R3); 0 keeps the workload's value")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


def _workload(name, seed):
    from lbm_workloads import fields
    return {"reactor": lambda: fields.reactor(seed=seed),
            "flame": lambda: fields.flame_1d(seed=seed),
            "channel": lambda: fields.channel_2d(seed=seed),
            "tube": lambda: fields.microtube(seed=seed),
            "box": lambda: fields.perturbed_box((128, 64, 64), "D3Q27", seed=seed,
                                                dx=12.5e-6, amp_u=1.0)}[name]()


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


def boundary_spec(w):
    """Boundary description of a workload (faces, inlet, outlet, walls,
    solid nodes), or None for a periodic box."""
    keys = ("faces", "inlet", "outlet", "wall_T", "solid", "solid_kind")
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
    workload (weak scaling); a node update is one lattice of one node, M + 2
    per node-step."""
    return nodes_per_rank * steps * world * (species + 2) / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling every 200 ms while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"],
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


def group_counters(group, workload, precision):
    """Per-node counters of a launch group from the committed ncu summary
    (profiles/group_counters.txt): {"fp32_flop", "fp64_flop", "dram_bytes"},
    or None when the summary has no line for it."""
    path = os.path.join(ROOT, "profiles", "group_counters.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if tuple(f[:3]) == (group, workload, precision):
            return {"fp32_flop": float(f[3]), "fp64_flop": float(f[4]),
                    "dram_bytes": float(f[5])}
    return None


def run_reference(args, rank):
    """The CPU oracle as it stands, on the same workload."""
    if rank != 0:
        return
    from lbm_workloads.mechanism import h2_air_synthetic
    from oracle import OracleLBM, thermo
    mech = h2_air_synthetic()
    w = _workload(args.workload, 0)
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], T_max=w["T_max"],
                  substeps=w["substeps"], boundaries=boundary_spec(w))
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    N = int(w["P"].size)
    M = mech.n_species
    v = N * args.steps * (M + 2) / dt
    line = {
        "impl": "reference", "metric": "node-updates/s", "value": v, "unit": "node-updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "nodes": N, "precision": "fp64",
                   "l2": "oracle on host cores"},
        "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} full steps of the workload after "
                                   f"{args.warmup} warm-up steps"},
        "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(args, w, mech, budget_s=15.0):
    """Oracle timed on the host on a bounded number of steps of the same workload."""
    from oracle import OracleLBM, thermo
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], T_max=w["T_max"],
                  substeps=w["substeps"], boundaries=boundary_spec(w))
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(args.steps, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    N = int(w["P"].size)
    return {"value": N * n * (mech.n_species + 2) / dt, "unit": "node-updates/s",
            "cores": 1, "kind": "oracle",
            "sample": f"{n} full steps of the workload (after 1 warm-up step), "
                      f"numpy single-threaded"}


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
    w = _workload(args.workload, seed=rank)
    if args.substeps:
        w["substeps"] = args.substeps
    N = int(w["P"].size)
    M = mech.n_species
    solver = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                        precision=args.precision, substeps=w["substeps"], T_max=w["T_max"],
                        device=local, **(boundary_spec(w) or {}))
    solver.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    info = solver.info
    state_bytes = 2 * info.L * info.Q * N * info.bytes_per_population
    flush = state_bytes < 2 * L2_BYTES
    flush_buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda") \
        if flush else None
    stream = torch.cuda.current_stream()

    solver.step(args.warmup)
    solver.synchronize()
    # kernel placement: the library's default for this grid and precision
    # (which matched the autotuner's choice on every workload measured), the
    # values given on the command line, or --autotune (trial steps on the
    # current state; the solve itself is not advanced)
    if args.autotune:
        launch = solver.autotune(trial_steps=3)
    else:
        solver.set_launch(args.chem_lanes or -1, args.collide_split)
        launch = solver.launch()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            if flush:
                flush_buf.zero_()
            starts[k].record(stream)
            solver.step(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
    solver.synchronize()
    total_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # per-kernel device times: a second pass of the same number of steps with
    # events around every launch group (lbm_step_timed), L2 flushed likewise
    kms = [0.0, 0.0]
    for k in range(args.steps):
        if flush:
            flush_buf.zero_()
        kms = lbm.lbm_step_timed(solver.h, 1, kms)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(total_ms, pg)
    if pg:
        pg.barrier()
    ms_per_step = total_ms / args.steps
    node_steps = N * args.steps * world
    # kernels per step: the moments with the reaction sub-steps (k_moments,
    # one thread per node, or k_mchem, chem_lanes lanes per node), the
    # collision (one kernel, or two when split); with interface nodes also
    # the boundary kernel and, after it on the side stream, the interface
    # nodes' sub-steps (k_chem)
    has_bnd = boundary_spec(w) is not None
    launches_per_step = 1 + (2 if has_bnd else 0) + (2 if launch["collide_split"] else 1)
    value = node_updates_per_s(N, args.steps, world, M, total_ms * 1e-3)

    # roofline of the dominant launch group.  Both paths are bound by
    # arithmetic, not by HBM: a node-step executes ~60k FP32 FLOP (mixed
    # path, float-float chemistry and Newton) or ~17k FP64 FLOP for ~2.2 /
    # 4.3 kB of populations, far above the machine balance (80.6 TFLOP/s FP32
    # or 1.25 FP64 against ~6.7 TB/s).  The ALU roof is the bound; the HBM
    # figures of the same group are reported beside it.
    names = launch_groups(launch, has_bnd)
    dom = int(np.argmax(kms))
    dom_ms = kms[dom] / args.steps
    alg_bytes = 2 * info.L * info.Q * info.bytes_per_population   # per node-step
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_gbs = alg_bytes * N / (dom_ms * 1e-3) / 1e9
    cnt = group_counters(names[dom], args.workload, args.precision)
    key = "fp64_flop" if args.precision == "fp64" else "fp32_flop"
    peak = FP64_PEAK_TFLOPS if args.precision == "fp64" else FP32_PEAK_TFLOPS
    achieved = cnt[key] * N / (dom_ms * 1e-3) / 1e12 if cnt else None
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if achieved else None,
            "traffic": cnt["dram_bytes"] * N if cnt else None, "kernel": names[dom],
            "flop_per_node": cnt[key] if cnt else None,
            "peak_source": ("nominal FP64 1.25 TFLOP/s (recipe); FMA probe measured 1.25"
                            if args.precision == "fp64" else
                            "FP32: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz (unit counts, "
                            "maximum clock)"),
            "hbm": {"achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_gbs / hbm_peak, "alg_bytes_per_node": alg_bytes,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback"}}

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
        e2e = {"value": node_updates_per_s(N, args.steps, world, M, e2e_s),
               "unit": "node-updates/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "timed": "init from host fields + K steps + all fields read back to host"}

    solver.close()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args, w, mech)
    line = {
        "metric": "node-updates/s", "value": value, "unit": "node-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64",
                  "fp32": "f32 (temperature Newton and chemistry in float-float)",
                  "fp16": "f16 offset storage, f32 arithmetic (temperature Newton and "
                          "chemistry in float-float)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "nodes": N, "lattice": w["lattice"],
                   "species": M, "precision": args.precision, "substeps": w["substeps"],
                   "node_steps_per_s": node_steps / (total_ms * 1e-3),
                   "l2": "256 MB buffer overwritten between timed steps" if flush
                   else "state larger than L2", "parallelism": f"replicas x{world}",
                   "launch": launch},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step * args.steps,
        "kernel_ms_per_step": {names[0]: kms[0] / args.steps, names[1]: kms[1] / args.steps},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
