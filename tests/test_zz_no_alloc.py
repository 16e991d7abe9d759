"""lbm_step_noalloc, the entry point for callers that cannot allocate device
memory (an application owning every device allocation, a loop that must not
synchronise on cudaMalloc, a fixed memory budget), must advance populations
exactly as lbm_step does.  It keeps its scratch in a fixed array inside the
library, so this file is collected last: a failure here leaves every other
test already run.  Both calls in a row are compared with the handle-based
path, within the FP64 parity tolerance of the other GPU tests."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

pytestmark = pytest.mark.gpu
RTOL_FP64 = 1e-10


def _rel_err(a, b):
    L = b.shape[0]
    return max(float(np.max(np.abs(a[l] - b[l])) / np.max(np.abs(b[l]))) for l in range(L))


def test_noalloc_step_matches_lbm_step_two_calls():
    import torch
    from paper_2108_07605_gb300 import build, lbm
    build.build()
    mech = h2_air_synthetic()
    w = fields.perturbed_box((10, 7, 5), "D3Q27", mech=mech)      # ragged: 350 nodes
    ref = lbm.Solver(mech, lattice="D3Q27", shape=w["shape"], dx=w["dx"], T_max=w["T_max"])
    ref.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    info = ref.info
    count = info.L * info.Q * ref.N
    pops = [torch.empty(count, dtype=torch.float64, device="cuda") for _ in range(2)]
    lbm.lbm_get_populations(ref.h, pops[0])
    T = torch.tensor(np.ascontiguousarray(w["T"]).reshape(-1), dtype=torch.float64,
                     device="cuda")
    torch.cuda.synchronize()
    cfg = ref.cfg                  # same configuration; its allocation hooks are ignored
    for k in range(2):
        lbm.lbm_step_noalloc(cfg, pops[k % 2], pops[(k + 1) % 2], T)
        ref.step(1)
        got = pops[(k + 1) % 2].cpu().numpy().reshape(info.L, info.Q, ref.N)
        want = ref.populations()
        assert _rel_err(got, want) < RTOL_FP64, (k, _rel_err(got, want))
    ref.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2108_07605_gb300 import lbm
    mech = h2_air_synthetic()
    cfg, _ = lbm.make_config(mech, shape=(64, 16, 17), use_torch_allocator=False)
    buf = torch.empty(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(cfg, buf, buf[4:], buf)
    assert e.value.status == 6
    assert "16384" in str(e.value)
