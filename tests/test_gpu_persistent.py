"""The batched step as ONE persistent launch over a work-list
(lbm_launch.persistent = 2): a grid of the resident blocks claims boundary,
moments, parameter and collision items of every domain in stage order, each
item waiting (boundedly) only for the items it reads.

* Uneven domains (flame with inlet and outlet, periodic box, staircase tube
  with off-grid wall targets, reactor; D2Q9 channel and box) advanced by a
  single-launch plan (split collision: parameter then collision items; fused:
  one collision item per node tile) equal the same handles stepped alone
  with the same placement: 1e-12 relative
  per lattice in FP64, 5e-5 in FP32 storage (float-float chemistry in the
  launch's dynamic shared memory), for 1, 2 and 4 nodes per thread, over odd
  and even step counts.
* A small mix equals the FP64 oracle element by element (1e-10).
* Many small domains at once (dependencies across 16 domains).
* The bounded wait the dependencies use ends on a set word at once and gives
  up on a word that nothing sets, raising the abort word.
* The plan autotuner may pick the single launch; whatever it picks agrees.
"""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, make_oracle, max_rel_err_per_lattice, oracle_populations

pytestmark = pytest.mark.gpu

# FP32: the separate steps run the same placement (one thread per node for
# the bulk chemistry), but their interface nodes take the float-float
# sub-steps with eight lanes each (another summation order), which the
# flame's steep front amplifies over seven steps to ~2e-5 of a lattice's
# largest population
TOL = {"fp64": 1e-12, "fp32": 5e-5}
# temperature (K): FP64 to its Newton tolerance; FP32 storage to well inside
# its stated 0.05 K against the oracle (FP32 moments summed in another order)
TOL_T = {"fp64": 3e-6, "fp32": 1e-3}


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _mix3d(mech):
    return [fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10),
            fields.perturbed_box((10, 7, 5), "D3Q27", mech=mech),
            fields.microtube(nx=10, ny=9, nz=9, radius=3.6, offgrid=True),
            fields.reactor(n=6)]


def _keep(a, w):
    return np.ones(a.N, bool) if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)


def _run_pairs(mech, ws, precision, npt, runs, split=1):
    from paper_2108_07605_gb300 import lbm
    pairs = [(make_gpu(mech, w, precision=precision), make_gpu(mech, w, precision=precision))
             for w in ws]
    plan = lbm.lbm_batch_create([a.h for a, _ in pairs])
    lbm.lbm_batch_set_launch(plan, collide_split=split, persistent=2, nodes_per_thread=npt)
    got = lbm.lbm_batch_get_launch(plan)
    assert got["persistent"] == 2 and got["nodes_per_thread"] == npt
    assert got["collide_split"] == split
    total = 0
    for r in runs:
        lbm.lbm_batch_run(plan, r)
        total += r
    lbm.lbm_batch_destroy(plan)
    for _, b in pairs:
        b.set_launch(chem_lanes=1, collide_split=split)
        b.step(total)
    return pairs


@pytest.mark.parametrize("precision,npt,split", [
    ("fp64", 1, 1), ("fp64", 2, 1), ("fp64", 4, 1), ("fp64", 1, 0), ("fp64", 2, 0),
    ("fp32", 1, 1), ("fp32", 4, 1), ("fp32", 1, 0)])
def test_single_launch_equals_separate_steps_d3q27(mech, precision, npt, split):
    ws = _mix3d(mech)
    pairs = _run_pairs(mech, ws, precision, npt, [3, 4], split)
    for (a, b), w in zip(pairs, ws):
        err = max_rel_err_per_lattice(a.populations(), b.populations(), _keep(a, w))
        assert np.all(err <= TOL[precision]), (w.get("name"), err.max())
        ta, tb = a.moments()["T"], b.moments()["T"]
        k = _keep(a, w)
        assert np.max(np.abs(ta.reshape(-1)[k] - tb.reshape(-1)[k])) <= TOL_T[precision]
        a.close()
        b.close()


@pytest.mark.parametrize("split", [1, 0])
def test_single_launch_equals_separate_steps_d2q9(mech, split):
    ws = [fields.channel_2d(nx=30, ny=9), fields.perturbed_box((17, 6, 1), "D2Q9", mech=mech)]
    pairs = _run_pairs(mech, ws, "fp64", 2, [5, 4], split)
    for a, b in pairs:
        err = max_rel_err_per_lattice(a.populations(), b.populations())
        assert np.all(err <= TOL["fp64"]), err.max()
        a.close()
        b.close()


def test_single_launch_many_domains(mech):
    """16 domains of different sizes: every collision item waits for its own
    domain's parameters, every parameter item for its domain's first stage."""
    ws = []
    for k in range(16):
        if k % 3 == 0:
            ws.append(fields.reactor(seed=k, n=4 + k % 5))
        elif k % 3 == 1:
            ws.append(fields.flame_1d(seed=k, nx=24 + 4 * k, ny=2, nz=2, x_ign=8))
        else:
            ws.append(fields.perturbed_box((6 + k % 4, 5, 4), "D3Q27", seed=k, mech=mech))
    pairs = _run_pairs(mech, ws, "fp64", 1, [2, 1])
    for (a, b), w in zip(pairs, ws):
        err = max_rel_err_per_lattice(a.populations(), b.populations(), _keep(a, w))
        assert np.all(err <= TOL["fp64"]), err.max()
        a.close()
        b.close()


@pytest.mark.parametrize("split", [1, 0])
def test_single_launch_matches_the_oracle(mech, split):
    """FP64, element by element against the oracle after 4 steps."""
    from paper_2108_07605_gb300 import lbm
    ws = [fields.flame_1d(nx=24, ny=2, nz=2, x_ign=6, mech=mech),
          fields.microtube(nx=8, ny=9, nz=9, radius=3.6, mech=mech, offgrid=True),
          fields.perturbed_box((7, 5, 4), "D3Q27", mech=mech)]
    gs = [make_gpu(mech, w) for w in ws]
    plan = lbm.lbm_batch_create([g.h for g in gs])
    lbm.lbm_batch_set_launch(plan, collide_split=split, persistent=2, nodes_per_thread=1)
    lbm.lbm_batch_run(plan, 4)
    lbm.lbm_batch_destroy(plan)
    for g, w in zip(gs, ws):
        o = make_oracle(mech, w)
        o.step(4)
        ref = oracle_populations(o)
        got = g.populations()
        keep = _keep(g, w)
        ref, got = ref[:, :, keep], got[:, :, keep]
        scale = np.max(np.abs(ref), axis=(1, 2), keepdims=True)
        assert np.all(np.abs(got - ref) <= 1e-10 * np.abs(ref) + 1e-13 * scale)
        g.close()


def test_single_launch_autotune(mech):
    from paper_2108_07605_gb300 import lbm
    ws = _mix3d(mech)
    pairs = [(make_gpu(mech, w), make_gpu(mech, w)) for w in ws]
    plan = lbm.lbm_batch_create([a.h for a, _ in pairs])
    chosen = lbm.lbm_batch_autotune(plan, 2)
    assert chosen["persistent"] in (0, 1, 2)
    assert chosen["nodes_per_thread"] in (1, 2, 4)
    lbm.lbm_batch_run(plan, 3)
    lbm.lbm_batch_destroy(plan)
    for (a, b), w in zip(pairs, ws):
        b.step(3)
        err = max_rel_err_per_lattice(a.populations(), b.populations(), _keep(a, w))
        assert np.all(err <= TOL["fp64"]), err.max()
        a.close()
        b.close()


def test_bounded_wait_probe():
    from paper_2108_07605_gb300 import lbm
    ok, abort, us = lbm.lbm_wait_probe(True, 2_000_000)
    assert ok == 1 and abort == 0 and us < 2_000
    ok, abort, us = lbm.lbm_wait_probe(False, 2_000_000)   # nothing sets the word
    assert ok == 0 and abort == 1
    assert 2_000 <= us < 1_000_000
    with pytest.raises(lbm.LBMError):
        lbm.lbm_wait_probe(False, 10 ** 9)                 # beyond the probe's limit
