"""lbm_batch_step: several handles of different sizes and boundary layouts
advanced by one launch per kernel per step must reproduce separate lbm_step
calls.  The per-node arithmetic is the same; the batched kernels are separate
instantiations, so the compiler may fuse multiply-adds differently and the
results agree to rounding: within 1e-12 relative per lattice in FP64 and
1e-5 in FP32 storage after 7-9 steps."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, max_rel_err_per_lattice

TOL = {"fp64": 1e-12, "fp32": 1e-5}

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _pair(mech, w, precision):
    return make_gpu(mech, w, precision=precision), make_gpu(mech, w, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_separate_steps_d3q27(mech, precision):
    from paper_2108_07605_gb300 import lbm
    ws = [fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10),
          fields.perturbed_box((10, 7, 5), "D3Q27", mech=mech),
          fields.microtube(nx=10, ny=9, nz=9, radius=3.6),
          fields.reactor(n=6)]
    pairs = [_pair(mech, w, precision) for w in ws]
    lbm.lbm_batch_step([a.h for a, _ in pairs], 7)
    for _, b in pairs:
        b.step(7)
    for (a, b), w in zip(pairs, ws):
        keep = np.ones(a.N, bool) if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
        err = max_rel_err_per_lattice(a.populations(), b.populations(), keep)
        assert np.all(err <= TOL[precision]), (w.get("name"), err.max())
        a.close()
        b.close()


def test_batch_equals_separate_steps_d2q9(mech):
    from paper_2108_07605_gb300 import lbm
    ws = [fields.channel_2d(nx=30, ny=9), fields.perturbed_box((17, 6, 1), "D2Q9", mech=mech)]
    pairs = [_pair(mech, w, "fp64") for w in ws]
    lbm.lbm_batch_step([a.h for a, _ in pairs], 5)
    lbm.lbm_batch_step([a.h for a, _ in pairs], 4)       # odd then even parity
    for _, b in pairs:
        b.step(9)
    for a, b in pairs:
        err = max_rel_err_per_lattice(a.populations(), b.populations())
        assert np.all(err <= TOL["fp64"]), err.max()
        a.close()
        b.close()


def test_batch_rejects_mixed_lattices(mech):
    from paper_2108_07605_gb300 import lbm
    a = make_gpu(mech, fields.reactor(n=4))
    b = make_gpu(mech, fields.channel_2d(nx=12, ny=5))
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_step([a.h, b.h], 1)
    assert e.value.status == 1
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_plan_graph_replay(mech, precision):
    """A captured plan (CUDA graphs) replays the batched step; odd step
    counts, and a handle advanced on its own between runs, keep it right."""
    from paper_2108_07605_gb300 import lbm
    ws = [fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10), fields.reactor(n=6)]
    pairs = [_pair(mech, w, precision) for w in ws]
    plan = lbm.lbm_batch_create([a.h for a, _ in pairs])
    lbm.lbm_batch_run(plan, 3)
    pairs[1][0].step(2)                 # outside the plan
    lbm.lbm_batch_run(plan, 4)
    lbm.lbm_batch_destroy(plan)
    pairs[0][1].step(7)
    pairs[1][1].step(9)
    for a, b in pairs:
        err = max_rel_err_per_lattice(a.populations(), b.populations())
        assert np.all(err <= TOL[precision]), err.max()
        a.close()
        b.close()
