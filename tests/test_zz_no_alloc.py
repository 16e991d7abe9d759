"""lbm_step_noalloc, the entry point for callers that cannot allocate device
memory (an application owning every device allocation, a loop that must not
synchronise on cudaMalloc, a fixed memory budget), must advance populations
exactly as lbm_step does.  It keeps its scratch in a fixed array inside the
library, so this file is collected last: a failure here leaves every other
test already run.  Each case makes two calls in a row and compares both with
the handle-based path: in the default placement of lbm_step within the FP64
parity tolerance of the other GPU tests, and in the placement the entry
point always uses (one thread per node, fused collision) bit for bit, FP32
storage included."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

pytestmark = pytest.mark.gpu
RTOL_FP64 = 1e-10


def _rel_err(a, b):
    L = b.shape[0]
    return max(float(np.max(np.abs(a[l] - b[l])) / np.max(np.abs(b[l]))) for l in range(L))


def _two_calls(shape, lattice, precision, same_placement):
    import torch
    from paper_2108_07605_gb300 import build, lbm
    build.build()
    mech = h2_air_synthetic()
    w = fields.perturbed_box(shape, lattice, mech=mech)
    ref = lbm.Solver(mech, lattice=lattice, shape=w["shape"], dx=w["dx"], T_max=w["T_max"],
                     precision=precision)
    if same_placement:
        ref.set_launch(1, 0)
    ref.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    info = ref.info
    count = info.L * info.Q * ref.N
    store = torch.float64 if precision == "fp64" else torch.float32
    pops = [torch.empty(count, dtype=store, device="cuda") for _ in range(2)]
    start = torch.empty(count, dtype=torch.float64, device="cuda")
    lbm.lbm_get_populations(ref.h, start)
    pops[0].copy_(start)           # FP32 storage: exact, the values are FP32 numbers
    T = torch.tensor(np.ascontiguousarray(w["T"]).reshape(-1), dtype=torch.float64,
                     device="cuda")
    torch.cuda.synchronize()
    cfg = ref.cfg                  # same configuration; its allocation hooks are ignored
    errs = []
    for k in range(2):
        lbm.lbm_step_noalloc(cfg, pops[k % 2], pops[(k + 1) % 2], T)
        ref.step(1)
        got = pops[(k + 1) % 2].double().cpu().numpy().reshape(info.L, info.Q, ref.N)
        want = ref.populations()
        errs.append(_rel_err(got, want))
    ref.close()
    return errs


def test_noalloc_step_matches_lbm_step_two_calls():
    errs = _two_calls((10, 7, 5), "D3Q27", "fp64", same_placement=False)   # ragged: 350 nodes
    assert max(errs) < RTOL_FP64, errs


@pytest.mark.parametrize("lattice,shape,precision", [
    ("D3Q27", (10, 7, 5), "fp64"),
    ("D3Q27", (10, 7, 5), "fp32"),
    ("D2Q9", (37, 11, 1), "fp32"),
])
def test_noalloc_step_equals_lbm_step_in_the_same_placement(lattice, shape, precision):
    errs = _two_calls(shape, lattice, precision, same_placement=True)
    assert max(errs) == 0.0, errs


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2108_07605_gb300 import lbm
    mech = h2_air_synthetic()
    shape = (64, 16, 17)                       # 17 408 nodes, above the 16 384 limit
    cfg, _ = lbm.make_config(mech, shape=shape, use_torch_allocator=False)
    N = 64 * 16 * 17
    count = (mech.n_species + 1) * 27 * N
    # buffers sized for the grid, so that only the library's own node-count
    # check stands between this call and a launch
    a = torch.zeros(count, dtype=torch.float64, device="cuda")
    b = torch.zeros(count, dtype=torch.float64, device="cuda")
    T = torch.full((N,), 300.0, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_step_noalloc(cfg, a, b, T)
    assert e.value.status == 6
    assert "16384" in str(e.value)


def test_noalloc_binding_rejects_undersized_and_host_buffers():
    import torch
    from paper_2108_07605_gb300 import lbm
    mech = h2_air_synthetic()
    cfg, _ = lbm.make_config(mech, shape=(4, 4, 4), use_torch_allocator=False)
    N = 64
    count = (mech.n_species + 1) * 27 * N
    good = torch.zeros(count, dtype=torch.float64, device="cuda")
    T = torch.full((N,), 300.0, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        lbm.lbm_step_noalloc(cfg, good, good[: count - 1], T)
    with pytest.raises(ValueError):
        lbm.lbm_step_noalloc(cfg, good.cpu(), good.clone(), T)
    with pytest.raises(ValueError):
        lbm.lbm_step_noalloc(cfg, good, good.float(), T)
