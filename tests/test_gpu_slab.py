"""The x-slab decomposition on the GPU, emulated in one process: two
library handles on the same GPU hold the two slabs of a domain (with their
halo planes), and before every step the halos are copied between them
(lbm_get_planes / lbm_set_planes, device to device; the copies run between
the handles' steps, never while a kernel of the other handle waits).  The
slabs' own planes equal the undivided domain's, bit for bit, in FP64 and
FP32 storage, and the flame diagnostics of the slabs' own planes combine
into the undivided domain's (the integral to summation order).  On several GPUs the same exchange runs as NCCL point-to-point
transfers (slab.Exchange); this run has one GPU."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic
from paper_2108_07605_gb300 import slab

from helpers import make_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["flame", "tube", "box"])
def test_two_slabs_equal_one_domain(case, precision):
    mech = h2_air_synthetic()
    if case == "flame":
        w = fields.flame_1d(nx=64, ny=4, nz=4, x_ign=16, mech=mech)
    elif case == "tube":
        w = fields.microtube(nx=40, ny=20, nz=20, radius=9.5, mech=mech, offgrid=True)
    else:
        w = fields.perturbed_box((32, 8, 8), "D3Q27", mech=mech)
    nsteps = 6
    whole = make_gpu(mech, w, precision=precision)
    whole.step(nsteps)
    ref = whole.populations()
    dref = whole.diagnostics()
    whole.close()
    layout = slab.SlabLayout(w["shape"][0], 2, w["faces"][0] == "periodic")
    parts = [make_gpu(mech, slab.slab_workload(w, layout, r), precision=precision)
             for r in range(2)]
    engines = [slab.SolverEngine(p) for p in parts]
    for _ in range(nsteps):
        slab.exchange_in_process(layout, engines)
        for e in engines:
            e.step(1)
    # the whole domain's diagnostics from the slabs' own planes (the
    # combination the ranks' all-gather performs)
    dg = slab.combine_diagnostics([slab.own_diagnostics(layout, r, engines[r], w["dx"])
                                   for r in range(2)])
    assert dg["hrr_integral"] == pytest.approx(dref["hrr_integral"], rel=1e-12)
    for k in ("hrr_max", "flame_x", "T_max", "u_max"):
        assert dg[k] == dref[k], k
    nx, ny, nz = w["shape"]
    L, Q = ref.shape[:2]
    ref = ref.reshape(L, Q, nz, ny, nx)
    solid = None if w.get("solid") is None else np.asarray(w["solid"])
    for r, p in enumerate(parts):
        x_lo, x_hi, g_lo, g_hi = layout.local(r)
        got = p.populations().reshape(L, Q, nz, ny, g_hi - g_lo)[..., x_lo - g_lo:x_hi - g_lo]
        want = ref[..., x_lo:x_hi]
        if solid is not None:
            keep = ~solid[..., x_lo:x_hi]
            got, want = got[:, :, keep], want[:, :, keep]
        assert np.array_equal(got, want), (r, float(np.max(np.abs(got - want))))
        p.close()
