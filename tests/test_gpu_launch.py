"""Kernel placement (moments and reaction sub-steps with one thread per node,
or with groups of 4 / 8 lanes per node; collision fused or split into a
per-node parameter kernel and a nine-threads-per-node direction kernel) and
the autotuner that chooses among them.

The placements evaluate the same formulas; only the species production rates
and the Newton polynomial's terms are summed in another order when the work
is dealt out over lanes, and
the compiler may fuse multiply-adds differently in the two collision
kernels, so they agree to rounding: 1e-13 relative per lattice in FP64.  In
FP32 storage the rounding differences of the first step grow through the
trace species' chemistry and the wall reconstruction of the staircase tube
(up to 1e-5 of a lattice's largest population after 10 steps), so the bound
there is 1e-4, far inside the FP32 path's field tolerances against the FP64
oracle.  The autotuner's trial steps leave the
handle's state untouched: a solve that was autotuned continues bit for bit
like one that was not, given the same placement.  Persistent grids for
batch plans (each block looping over work-list tiles) change only which
block updates a tile, so a plan gives bit-identical results with and
without them."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, max_rel_err_per_lattice, perturbed_box

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-13, "fp32": 1e-4}
PLACEMENTS = [(1, 0), (4, 0), (8, 0), (1, 1), (4, 1), (8, 1)]


def _pl(cl, cs, persistent=0):
    return {"chem_lanes": cl, "collide_split": cs, "persistent": persistent,
            "nodes_per_thread": 1}


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _cases(mech):
    flame = fields.flame_1d(seed=2, nx=48, ny=4, nz=4, x_ign=12, mech=mech)
    chan = fields.channel_2d(seed=4, nx=40, ny=10, mech=mech)
    box = perturbed_box((9, 6, 5), "D3Q27", mech=mech)      # 270 nodes: a ragged k_coll block
    tube = fields.microtube(seed=6, nx=12, ny=10, nz=10, radius=4.5, mech=mech)
    return [("flame", flame), ("channel", chan), ("box", box), ("tube", tube)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_placements_agree(mech, precision):
    for name, w in _cases(mech):
        got = []
        for cl, cs in PLACEMENTS:
            g = make_gpu(mech, w, precision=precision)
            g.set_launch(cl, cs)
            assert g.launch() == _pl(cl, cs)
            g.step(10)
            got.append(g.populations())
            g.close()
        mask = None
        if w.get("solid") is not None:
            mask = ~np.asarray(w["solid"], bool).reshape(-1)
        for k in range(1, len(got)):
            err = max_rel_err_per_lattice(got[k], got[0], mask)
            assert np.all(err < TOL[precision]), (name, PLACEMENTS[k], err)


def test_default_placement_follows_grid_size(mech):
    small = make_gpu(mech, perturbed_box((8, 8, 8), "D3Q27", mech=mech), precision="fp32")
    assert small.launch() == _pl(4, 1)
    small.set_launch(1, 0)
    assert small.launch() == _pl(1, 0)
    small.set_launch(-1, -1)
    assert small.launch() == _pl(4, 1)
    small.close()
    small64 = make_gpu(mech, perturbed_box((8, 8, 8), "D3Q27", mech=mech))
    assert small64.launch() == _pl(1, 1)
    small64.close()
    big = make_gpu(mech, fields.reactor(seed=1, n=48, mech=mech), precision="fp32")
    assert big.launch() == _pl(1, 1)     # 110,592 nodes
    big.close()


def test_invalid_placement_rejected(mech):
    from paper_2108_07605_gb300 import lbm
    g = make_gpu(mech, perturbed_box((4, 4, 4), "D3Q27", mech=mech))
    for cl, cs, p in [(2, 0, 0), (0, 0, 0), (4, 2, 0), (16, -1, 0), (1, 1, 2), (4, 0, -2)]:
        with pytest.raises(lbm.LBMError):
            g.set_launch(cl, cs, p)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_leaves_the_solve_unchanged(mech, precision):
    w = fields.flame_1d(seed=5, nx=40, ny=4, nz=4, x_ign=10, mech=mech)
    a = make_gpu(mech, w, precision=precision)
    a.step(3)
    chosen = a.autotune(trial_steps=2)
    assert (chosen["chem_lanes"], chosen["collide_split"]) in PLACEMENTS
    assert chosen["persistent"] == 0
    assert a.launch() == chosen
    a.step(6)
    b = make_gpu(mech, w, precision=precision)       # the same history, untuned
    b.step(3)
    b.set_launch(chosen["chem_lanes"], chosen["collide_split"])
    b.step(6)
    pa, pb = a.populations(), b.populations()
    ma, mb = a.moments(), b.moments()
    a.close()
    b.close()
    assert np.array_equal(pa, pb)
    assert np.array_equal(ma["T"], mb["T"])


def test_batch_autotune_then_run_matches_separate_solves(mech):
    from paper_2108_07605_gb300 import lbm
    ws = [fields.reactor(seed=7, n=6, mech=mech),
          perturbed_box((7, 5, 4), "D3Q27", mech=mech),
          fields.flame_1d(seed=8, nx=32, ny=4, nz=4, x_ign=8, mech=mech)]
    batched = [make_gpu(mech, w) for w in ws]
    plan = lbm.lbm_batch_create([g.h for g in batched])
    chosen = lbm.lbm_batch_autotune(plan, trial_steps=2)
    assert (chosen["chem_lanes"], chosen["collide_split"]) in PLACEMENTS
    lbm.lbm_batch_run(plan, 5)
    lbm.lbm_batch_destroy(plan)
    for g, w in zip(batched, ws):
        s = make_gpu(mech, w)
        s.set_launch(chosen["chem_lanes"], chosen["collide_split"])
        s.step(5)
        err = max_rel_err_per_lattice(g.populations(), s.populations())
        s.close()
        g.close()
        assert np.all(err < 1e-12), err


def test_persistent_batched_grids_match(mech):
    """A 40^3 reactor puts about 2,000 tiles on the collision work-list, more
    than the GPU holds at once, so the persistent blocks loop several times."""
    from paper_2108_07605_gb300 import lbm
    ws = [fields.reactor(seed=9, n=40, mech=mech),
          perturbed_box((9, 6, 5), "D3Q27", mech=mech),
          fields.flame_1d(seed=10, nx=64, ny=4, nz=4, x_ign=16, mech=mech)]
    out = {}
    for persistent in (0, 1):
        gs = [make_gpu(mech, w) for w in ws]
        plan = lbm.lbm_batch_create([g.h for g in gs])
        lbm.lbm_batch_set_launch(plan, 1, 1, persistent)
        assert lbm.lbm_batch_get_launch(plan) == _pl(1, 1, persistent)
        lbm.lbm_batch_run(plan, 4)
        lbm.lbm_batch_destroy(plan)
        out[persistent] = [g.populations() for g in gs]
        for g in gs:
            g.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)
