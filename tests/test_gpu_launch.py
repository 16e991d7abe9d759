"""Kernel placement of the reaction sub-steps (thread per node inside the
moments kernel, or one warp per node in their own kernel) and the
autotuner that chooses between them.

Both placements evaluate the same rate formulas in the same order, so they
agree to rounding: 1e-13 relative per lattice in FP64, 1e-5 in FP32 storage
(the batching tolerance).  The autotuner's trial steps leave the handle's
state untouched: a solve that was autotuned continues bit for bit like one
that was not, given the same placement."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, max_rel_err_per_lattice, perturbed_box

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-13, "fp32": 1e-5}


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _cases(mech):
    flame = fields.flame_1d(seed=2, nx=48, ny=4, nz=4, x_ign=12, mech=mech)
    chan = fields.channel_2d(seed=4, nx=40, ny=10, mech=mech)
    box = perturbed_box((9, 6, 5), "D3Q27", mech=mech)
    return [("flame", flame), ("channel", chan), ("box", box)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chemistry_placements_agree(mech, precision):
    for name, w in _cases(mech):
        got = []
        for cpw in (0, 1):
            g = make_gpu(mech, w, precision=precision)
            g.set_launch(cpw)
            assert g.launch()["chem_per_warp"] == cpw
            g.step(10)
            got.append(g.populations())
            g.close()
        err = max_rel_err_per_lattice(got[1], got[0])
        assert np.all(err < TOL[precision]), (name, err)


def test_default_placement_follows_grid_size(mech):
    small = make_gpu(mech, perturbed_box((8, 8, 8), "D3Q27", mech=mech))
    assert small.launch()["chem_per_warp"] == 1
    small.set_launch(0)
    assert small.launch()["chem_per_warp"] == 0
    small.set_launch(-1)
    assert small.launch()["chem_per_warp"] == 1
    small.close()
    big = make_gpu(mech, fields.reactor(seed=1, n=48, mech=mech))   # 110,592 nodes
    assert big.launch()["chem_per_warp"] == 0
    big.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autotune_leaves_the_solve_unchanged(mech, precision):
    w = fields.flame_1d(seed=5, nx=40, ny=4, nz=4, x_ign=10, mech=mech)
    a = make_gpu(mech, w, precision=precision)
    a.step(3)
    chosen = a.autotune(trial_steps=2)
    assert chosen["chem_per_warp"] in (0, 1)
    assert a.launch() == chosen
    a.step(6)
    b = make_gpu(mech, w, precision=precision)
    b.set_launch(chosen["chem_per_warp"])
    b.step(9)
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
    assert chosen["chem_per_warp"] in (0, 1)
    lbm.lbm_batch_run(plan, 5)
    lbm.lbm_batch_destroy(plan)
    for g, w in zip(batched, ws):
        s = make_gpu(mech, w)
        s.set_launch(chosen["chem_per_warp"])
        s.step(5)
        err = max_rel_err_per_lattice(g.populations(), s.populations())
        s.close()
        g.close()
        assert np.all(err < 1e-12), err
