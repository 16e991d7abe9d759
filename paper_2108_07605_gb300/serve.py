"""Continuous-batching request loop for independent reactive-flow solves.

    python -m paper_2108_07605_gb300.serve [--requests 64] [--seed 0]
        [--budget-gb 40] [--chunk 100] [--precision fp32] [--step-scale 1.0]
    python -m paper_2108_07605_gb300.serve --plan-study [--precision fp64]
        (batch-plan placements timed on groups of the mix; plan_study)

Requests (reactor, flame or channel solves of different grid sizes) arrive
over time.  The loop admits a request as soon as it has arrived and its
device memory (lbm_bytes_required) fits the remaining budget, initialises
its populations on the GPU and keeps them resident.  Every tick advances a
set of resident requests together (policy "srpt", the default: those with
the least remaining work, up to a node count that fills the GPU; policy
"fifo": all of them): the advanced requests that share a lattice form a
batch plan (lbm_batch_create: the batched kernels - one launch per kernel
per step over the tiles of every request - captured as CUDA graphs), kept
while the set does not change and replayed for a chunk of steps no longer
than the shortest remaining request, so no request runs past its step
count.  The host waits only for the previous tick's event, never for the
whole device, so the next tick's launches are queued while one runs.  A request that has completed its steps is read back
(lbm_moments), its handle destroyed and its memory returned, and waiting
requests are admitted at the next tick.  An optional cap on the resident
nodes (max_nodes) admits in arrival order only while the resident requests'
nodes stay below it (a request larger than the cap runs alone): enough
resident work to fill the GPU, but not so much that every request advances
at the pace of all of them and finishes near the end.  A request whose solve fails (a
sticky device error such as a temperature Newton failure) is reported as
failed with the library's message; the others are unaffected.  Reported:
time-to-result (completion minus arrival) p50/p99 over the completed requests
and aggregate node-updates/s.

All arithmetic runs in the CUDA library; this module only schedules.
"""
import argparse
import json
import time

import numpy as np

from . import lbm


def _bc_kwargs(w):
    keys = ("faces", "inlet", "outlet", "wall_T", "solid", "solid_kind")
    if all(f == "periodic" for f in w.get("faces", ("periodic",) * 6)) and w.get("solid") is None:
        return {}
    return {k: w[k] for k in keys if k in w}


class Request:
    def __init__(self, rid, arrival, workload):
        self.rid = rid
        self.arrival = arrival
        self.w = workload
        self.remaining = int(workload["steps"])
        self.solver = None
        self.bytes = 0
        self.admitted = None
        self.finished = None
        self.result = None
        self.error = None

    @property
    def nodes(self):
        return int(self.w["P"].size)


class _TickFence:
    """Keeps the host at most one tick ahead of the GPU: an event is
    recorded on the current stream after each tick's launches, and the host
    waits for the previous tick's event (not for the whole device)."""

    def __init__(self, device):
        import torch
        self.torch, self.device = torch, device
        self.prev = None

    def mark(self):
        ev = self.torch.cuda.Event()
        ev.record(self.torch.cuda.current_stream(self.device))
        if self.prev is not None:
            self.prev.synchronize()
        self.prev = ev

    def drain(self):
        if self.prev is not None:
            self.prev.synchronize()
        self.prev = None


class Server:
    """Admission by device memory, continuous batching by lattice/precision.

    policy "srpt" (default): every arrived request that fits the memory
    budget is admitted and initialised at once (its populations stay
    resident); each tick advances the resident requests with the least
    remaining work (nodes x remaining steps) first, as many as keep the
    advanced nodes within active_nodes (at least one request): short
    requests do not wait behind long ones, and the GPU stays full.
    policy "fifo": every resident request advances every tick; admission in
    arrival order, optionally capped at max_nodes resident nodes."""

    def __init__(self, mech, budget_bytes, chunk=100, precision="fp32", device=0,
                 max_nodes=0, policy="srpt", active_nodes=600_000):
        if policy not in ("srpt", "fifo"):
            raise ValueError(policy)
        self.mech = mech
        # the library's fixed lbm_step_noalloc scratch is resident on the
        # device as soon as the library is loaded: it counts against the budget
        self.budget = int(budget_bytes) - lbm.NOALLOC_SCRATCH_BYTES
        self.max_nodes = int(max_nodes)   # 0: no cap on resident nodes (fifo)
        self.used = 0
        self.chunk = int(chunk)
        self.precision = precision
        self.device = device
        self.policy = policy
        self.active_nodes = int(active_nodes)

    def _config_bytes(self, req):
        cfg, _keep = lbm.make_config(self.mech, lattice=req.w["lattice"], shape=req.w["shape"],
                                     dx=req.w["dx"], precision=self.precision,
                                     substeps=req.w["substeps"], T_max=req.w["T_max"],
                                     use_torch_allocator=False, stream=0,
                                     **_bc_kwargs(req.w))
        return lbm.lbm_bytes_required(cfg)

    def _admit(self, req, now):
        w = req.w
        req.solver = lbm.Solver(self.mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                                precision=self.precision, substeps=w["substeps"],
                                T_max=w["T_max"], device=self.device, **_bc_kwargs(w))
        req.solver.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
        req.admitted = now
        self.used += req.bytes

    def _advanced(self, resident):
        """The requests this tick advances."""
        if self.policy == "fifo":
            return list(resident)
        order = sorted(resident, key=lambda r: (r.nodes * r.remaining, r.arrival, r.rid))
        chosen, nodes = [], 0
        for r in order:
            if chosen and nodes + r.nodes > self.active_nodes:
                continue
            chosen.append(r)
            nodes += r.nodes
        return chosen

    def run(self, stream, clock=time.perf_counter, on_tick=None):
        """stream: [(arrival_s, workload), ...] sorted by arrival.  Returns the
        finished requests (with .result = moments) in completion order."""
        pending = [Request(k, a, w) for k, (a, w) in enumerate(stream)]
        for r in pending:
            r.bytes = self._config_bytes(r)
            if r.bytes > self.budget:
                raise ValueError(f"request {r.rid} needs {r.bytes} B, above the budget")
        resident, done = [], []
        plans = {}          # (lattice, member ids) -> plan
        fence = _TickFence(self.device)
        t0 = clock()
        node_updates = 0
        while pending or resident:
            now = clock() - t0
            while pending and pending[0].arrival <= now and \
                    self.used + pending[0].bytes <= self.budget and \
                    (self.policy != "fifo" or self.max_nodes <= 0 or not resident or
                     sum(r.nodes for r in resident) + pending[0].nodes <= self.max_nodes):
                r = pending.pop(0)
                self._admit(r, now)
                resident.append(r)
            if not resident:
                if pending:
                    time.sleep(max(0.0, min(0.005, pending[0].arrival - now)))
                continue
            adv = self._advanced(resident)
            n = min(self.chunk, min(r.remaining for r in adv))
            groups = {}
            for r in adv:
                groups.setdefault(r.w["lattice"], []).append(r)
            for lat, grp in groups.items():
                key = (lat, tuple(r.rid for r in grp))
                if key not in plans:
                    plans[key] = lbm.lbm_batch_create([r.solver.h for r in grp])
                lbm.lbm_batch_run(plans[key], n)
                for r in grp:
                    r.remaining -= n
                    node_updates += n * r.nodes * (self.mech.n_species + 2)
            fence.mark()
            finished = [r for r in adv if r.remaining == 0]
            if finished:
                gone = {r.rid for r in finished}
                for key in [k for k in plans if gone & set(k[1])]:
                    lbm.lbm_batch_destroy(plans.pop(key))   # a plan must not outlive its handles
                for r in finished:
                    self._finish(r, clock, t0)
                    self.used -= r.bytes
                    done.append(r)
                resident = [r for r in resident if r.rid not in gone]
            # plans of member sets that no longer run are dropped
            live = {(lat, tuple(r.rid for r in grp)) for lat, grp in groups.items()}
            for key in [k for k in plans if k not in live]:
                lbm.lbm_batch_destroy(plans.pop(key))
            if on_tick:
                on_tick(clock() - t0, resident, pending, done)
        fence.drain()
        for plan in plans.values():
            lbm.lbm_batch_destroy(plan)
        self.elapsed = clock() - t0
        self.node_updates = node_updates
        return done

    @staticmethod
    def _finish(r, clock, t0):
        try:
            r.result = r.solver.moments()
        except lbm.LBMError as e:
            r.error = str(e)
        r.finished = clock() - t0
        try:
            r.solver.close()
        except lbm.LBMError:
            pass
        r.solver = None


def run_serial(mech, stream, budget, precision, device=0):
    """The baseline of the serving loop: the same requests one after another
    in arrival order, each advanced alone with lbm_step for its whole step
    count.  Returns summarize()'s dict."""
    import torch
    t0 = time.perf_counter()
    srv = Server(mech, budget, precision=precision, device=device)
    done = []
    node_updates = 0
    for k, (arr, w) in enumerate(stream):
        r = Request(k, arr, w)
        now = time.perf_counter() - t0
        if now < arr:
            time.sleep(arr - now)
        srv._admit(r, time.perf_counter() - t0)
        r.solver.step(r.remaining)
        torch.cuda.synchronize(device)
        node_updates += r.remaining * r.nodes * (mech.n_species + 2)
        Server._finish(r, time.perf_counter, t0)
        done.append(r)
    return summarize(done, time.perf_counter() - t0, node_updates)


def summarize(done, elapsed, node_updates):
    ok = [r for r in done if r.error is None]
    ttr = np.array([r.finished - r.arrival for r in ok]) if ok else np.array([np.nan])
    return {
        "requests": len(done),
        "failed": [{"request": r.rid, "kind": r.w.get("kind"), "error": r.error}
                   for r in done if r.error is not None],
        "p50_time_to_result_s": float(np.percentile(ttr, 50)),
        "p99_time_to_result_s": float(np.percentile(ttr, 99)),
        "mean_time_to_result_s": float(ttr.mean()),
        "makespan_s": float(elapsed),
        "node_updates_per_s": float(node_updates / elapsed),
        "node_updates": int(node_updates),
    }


# placements of a batch plan timed by plan_study: name -> lbm_batch_set_launch
# arguments (p0: one launch per kernel; p1: the same on persistent grids;
# p2: the whole step as one launch, nN = nodes per thread, f = fused
# collision)
PLAN_PLACEMENTS = {
    "p0": dict(persistent=0), "p0 fused": dict(persistent=0, collide_split=0, chem_lanes=1),
    "p1": dict(persistent=1),
    "p2 n1": dict(persistent=2, collide_split=1, nodes_per_thread=1),
    "p2 n2": dict(persistent=2, collide_split=1, nodes_per_thread=2),
    "p2 n4": dict(persistent=2, collide_split=1, nodes_per_thread=4),
    "p2 f n1": dict(persistent=2, collide_split=0, nodes_per_thread=1),
    "p2 f n2": dict(persistent=2, collide_split=0, nodes_per_thread=2),
}


def plan_study(mech, precision, device=0, steps=20, warmup=4, reps=3):
    """Batch-plan placements on groups of the serving mix (seed 0): small8,
    its first eight D3Q27 requests of at most 40 000 nodes; mixed, its
    first twelve D3Q27 requests; tube, the 600x40x40 microtube alone (also
    timed with lbm_step).  Per group: ms per step of every placement (best of
    `reps` runs of `steps` steps after `warmup`, host clock around
    lbm_batch_run and a device synchronize) and the autotuner's pick.
    Yields one dict per group."""
    import torch
    from lbm_workloads.fields import microtube, serving_mix
    stream = serving_mix(seed=0, n_requests=64, mech=mech)
    d3 = [w for _, w in stream if w["lattice"] == "D3Q27"]
    groups = {"small8": [w for w in d3 if int(np.prod(w["shape"])) <= 40000][:8],
              "mixed": d3[:12], "tube": [microtube(mech=mech)]}

    def solver(w):
        s = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                       precision=precision, substeps=w["substeps"], T_max=w["T_max"],
                       device=device, **_bc_kwargs(w))
        s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
        return s

    def timed(run):
        run(warmup)
        torch.cuda.synchronize(device)
        best = float("inf")
        for _ in range(reps):
            t0 = time.perf_counter()
            run(steps)
            torch.cuda.synchronize(device)
            best = min(best, (time.perf_counter() - t0) / steps)
        return best * 1e3

    for name, ws in groups.items():
        ss = [solver(w) for w in ws]
        out = {"group": name, "precision": precision, "domains": len(ss),
               "nodes": int(sum(s.N for s in ss)), "ms_per_step": {}}
        if len(ss) == 1:
            out["ms_per_step"]["lbm_step"] = timed(ss[0].step)
        plan = lbm.lbm_batch_create([s.h for s in ss])
        for pname, kw in PLAN_PLACEMENTS.items():
            lbm.lbm_batch_set_launch(plan, **kw)
            out["ms_per_step"][pname] = timed(lambda n: lbm.lbm_batch_run(plan, n))
        out["autotune"] = lbm.lbm_batch_autotune(plan, 3)
        lbm.lbm_batch_destroy(plan)
        for s in ss:
            s.close()
        yield out


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--requests", type=int, default=64)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--budget-gb", type=float, default=40.0)
    p.add_argument("--chunk", type=int, default=100)
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--step-scale", type=float, default=1.0,
                   help="multiply every request's step count (1.0 = the stated 1k-10k)")
    p.add_argument("--serial", action="store_true",
                   help="one request at a time (no batching), for comparison")
    p.add_argument("--max-nodes", type=int, default=0,
                   help="fifo: cap on the resident requests' nodes (0: admit by memory only)")
    p.add_argument("--policy", default="srpt", choices=["srpt", "fifo"])
    p.add_argument("--plan-study", action="store_true",
                   help="time the batch-plan placements on groups of the mix instead")
    p.add_argument("--active-nodes", type=int, default=600_000,
                   help="srpt: nodes advanced per tick (least remaining work first)")
    args = p.parse_args()
    from . import build
    build.build()
    from lbm_workloads.fields import serving_mix
    from lbm_workloads.mechanism import h2_air_synthetic
    mech = h2_air_synthetic()
    if args.plan_study:
        for out in plan_study(mech, args.precision):
            print(json.dumps(out), flush=True)
        return
    stream = serving_mix(seed=args.seed, n_requests=args.requests, mech=mech)
    for _, w in stream:
        w["steps"] = max(1, int(round(w["steps"] * args.step_scale)))
    budget = int(args.budget_gb * 1e9)
    if args.serial:
        out = run_serial(mech, stream, budget, args.precision)
    else:
        srv = Server(mech, budget, chunk=args.chunk, precision=args.precision,
                     max_nodes=args.max_nodes, policy=args.policy,
                     active_nodes=args.active_nodes)
        done = srv.run(stream)
        out = summarize(done, srv.elapsed, srv.node_updates)
    out.update(mode="serial" if args.serial else f"continuous batching ({args.policy})",
               precision=args.precision, step_scale=args.step_scale, seed=args.seed,
               chunk=args.chunk, budget_gb=args.budget_gb, max_nodes=args.max_nodes,
               active_nodes=args.active_nodes)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
