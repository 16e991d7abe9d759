"""The serving loop: requests that arrive while others run are admitted as
memory frees up, advanced together by batched steps, and each result equals
the same request solved alone within the batching tolerance (the batched
kernels do the same per-node arithmetic; results agree to rounding:
1e-12 relative in FP64, 1e-5 in FP32 storage)."""
import numpy as np
import pytest

from lbm_workloads.fields import serving_mix
from lbm_workloads.mechanism import h2_air_synthetic

pytestmark = pytest.mark.gpu


def _small_mix(mech, n=6):
    stream = serving_mix(seed=3, n_requests=n, mean_interarrival=0.01, steps=(20, 60),
                         max_nodes=64 * 8 * 8, mech=mech)
    out = []
    for arr, w in stream:
        # shrink grids so the test runs in seconds
        kind = w["kind"]
        from lbm_workloads import fields
        if kind == "reactor":
            w2 = fields.reactor(seed=w["seed"], n=8, mech=mech)
        elif kind == "flame":
            w2 = fields.flame_1d(seed=w["seed"], nx=64, ny=4, nz=4, x_ign=16, mech=mech)
        else:
            w2 = fields.channel_2d(seed=w["seed"], nx=40, ny=10, mech=mech)
        w2["steps"] = w["steps"]
        w2["kind"] = kind
        out.append((arr, w2))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_results_alone_equal_results_in_the_mix(precision):
    from paper_2108_07605_gb300 import lbm, serve
    mech = h2_air_synthetic()
    stream = _small_mix(mech)
    used = []
    srv = serve.Server(mech, budget_bytes=int(2e9), chunk=7, precision=precision)
    done = srv.run(stream, on_tick=lambda now, act, pend, fin: used.append(srv.used))
    assert len(done) == len(stream)
    for r in done:
        assert r.error is None, r.error
        w = r.w
        alone = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                           precision=precision, substeps=w["substeps"], T_max=w["T_max"],
                           **serve._bc_kwargs(w))
        alone.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
        alone.step(w["steps"])
        m = alone.moments()
        alone.close()
        tol = 1e-12 if precision == "fp64" else 1e-5
        for key in ("rho", "T", "Y"):
            scale = np.max(np.abs(m[key]))
            assert np.max(np.abs(m[key] - r.result[key])) <= tol * scale, (r.rid, key)
        umax = max(np.max(np.abs(m["u"])), 1e-30)
        assert np.max(np.abs(m["u"] - r.result["u"])) <= 1e3 * tol * umax, r.rid
    assert max(used) <= srv.budget


def test_admission_waits_for_memory():
    """With room for one request at a time, requests queue and still all
    finish; resident memory never exceeds the budget."""
    from paper_2108_07605_gb300 import serve
    mech = h2_air_synthetic()
    stream = _small_mix(mech, n=4)
    srv = serve.Server(mech, budget_bytes=1, chunk=10, precision="fp32")
    need = max(srv._config_bytes(serve.Request(0, a, w)) for a, w in stream)
    srv.budget = need
    resident = []
    done = srv.run(stream, on_tick=lambda now, act, pend, fin: resident.append(len(act)))
    assert len(done) == 4
    assert all(r.error is None for r in done)
    assert max(resident) <= 1 + 0        # one at a time fits
    assert srv.used == 0


def test_node_cap_admits_in_order_below_the_cap():
    """With a cap on resident nodes, the resident requests' nodes stay below
    it (one request at a time when a single one exceeds it) and every request
    still finishes."""
    from paper_2108_07605_gb300 import serve
    mech = h2_air_synthetic()
    stream = _small_mix(mech, n=6)
    cap = max(int(w["P"].size) for _a, w in stream)
    srv = serve.Server(mech, budget_bytes=int(2e9), chunk=10, precision="fp32", max_nodes=cap)
    resident = []
    done = srv.run(stream, on_tick=lambda now, act, pend, fin:
                   resident.append((len(act), sum(r.nodes for r in act))))
    assert len(done) == 6 and all(r.error is None for r in done)
    assert all(nodes <= cap or n == 1 for n, nodes in resident)

