"""Measurement studies behind the profiles/ summaries (not a test module).

    python tests/studies.py precision   # FP16 / FP32 field errors (profiles/precision_tube.md)
    python tests/studies.py placement   # kernel placements (profiles/placement_study.md)

Each prints one JSON line per measurement.  Needs a GPU and the built
library; the precision study also runs the CPU oracle on the small cases.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)
sys.path.insert(0, HERE)


def _errors(mg, mo, keep, M, D):
    return dict(
        Y=float(np.abs(mg["Y"] - mo["Y"].reshape(M, -1))[:, keep].max()),
        T=float(np.abs(mg["T"] - mo["T"].reshape(-1))[keep].max()),
        u=float(np.abs(mg["u"][:D] - mo["u"].reshape(mo["u"].shape[0], -1)[:D])[:, keep].max()),
        rho=float((np.abs(mg["rho"] - mo["rho"].reshape(-1)) / mo["rho"].reshape(-1))[keep].max()))


def precision():
    from lbm_workloads import fields
    from lbm_workloads.mechanism import h2_air_synthetic
    from helpers import make_gpu, make_oracle
    mech = h2_air_synthetic()
    M = mech.n_species
    cases = {
        "periodic box 10x7x5": (lambda: fields.perturbed_box((10, 7, 5), "D3Q27", mech=mech), 12),
        "flame layout 40x3x2": (lambda: fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10), 50),
        "channel 30x9": (lambda: fields.channel_2d(nx=30, ny=9), 50),
        "tube 10x9x9": (lambda: fields.microtube(nx=10, ny=9, nz=9, radius=3.6), 30),
        "flame 1024x4x4": (lambda: fields.flame_1d(), 20),
    }
    for name, (make, nsteps) in cases.items():
        w = make()
        o = make_oracle(mech, w)
        o.step(nsteps)
        mo = o.moments()
        keep = np.ones(w["P"].size, bool) if w.get("solid") is None \
            else ~np.asarray(w["solid"]).reshape(-1)
        for prec in ("fp32", "fp16"):
            g = make_gpu(mech, w, precision=prec)
            g.step(nsteps)
            e = _errors(g.moments(), mo, keep, M, o.vs.dim)
            g.close()
            print(json.dumps({"case": name, "reference": "oracle", "precision": prec,
                              "steps": nsteps, **e}), flush=True)
    w = fields.microtube()
    keep = ~np.asarray(w["solid"]).reshape(-1)
    res = {}
    for prec in ("fp64", "fp32", "fp16"):
        g = make_gpu(mech, w, precision=prec)
        t0 = time.time()
        g.step(200)
        g.synchronize()
        dt = time.time() - t0
        res[prec] = g.moments()
        g.close()
        print(json.dumps({"case": "tube 600x40x40", "precision": prec, "seconds_200_steps":
                          round(dt, 3)}), flush=True)
    for prec in ("fp32", "fp16"):
        e = _errors(res[prec], res["fp64"], keep, M, 3)
        print(json.dumps({"case": "tube 600x40x40", "reference": "FP64 GPU", "precision": prec,
                          "steps": 200, **e}), flush=True)


def placement():
    import torch
    import bench
    from paper_2108_07605_gb300 import lbm
    from lbm_workloads.mechanism import h2_air_synthetic
    from lbm_workloads import fields
    mech = h2_air_synthetic()
    for prec in ("fp32", "fp64"):
        for wl in ("flame", "flame256x32x32", "box"):
            # the largest flame of the serving mix (262 144 nodes) between the
            # 16 384-node flame and the 524 288-node box
            w = fields.flame_1d(seed=0, nx=256, ny=32, nz=32, x_ign=64, mech=mech) \
                if wl == "flame256x32x32" else bench._workload(wl, seed=0)
            s = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                           precision=prec, substeps=w["substeps"], T_max=w["T_max"],
                           **(bench.boundary_spec(w) or {}))
            s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
            s.step(3)
            n = 10 if wl == "flame" else 3
            for cl, cs in [(1, 0), (4, 0), (8, 0), (1, 1), (4, 1), (8, 1)]:
                s.set_launch(cl, cs)
                s.step(2)
                s.synchronize()
                kms = lbm.lbm_step_timed(s.h, n, [0.0, 0.0])
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                s.step(n)
                b.record()
                torch.cuda.synchronize()
                print(json.dumps({"precision": prec, "workload": wl, "chem_lanes": cl,
                                  "collide_split": cs, "moments_ms": kms[0] / n,
                                  "collision_ms": kms[1] / n,
                                  "step_ms": a.elapsed_time(b) / n}), flush=True)
            print(json.dumps({"precision": prec, "workload": wl,
                              "autotune": s.autotune(3)}), flush=True)
            s.close()


if __name__ == "__main__":
    import __graft_entry__
    __graft_entry__.build()
    {"precision": precision, "placement": placement}[sys.argv[1]]()
