"""GPU parity: the CUDA library (called through the C ABI) against the CPU
oracle on identical seeded inputs.

Tolerance of the FP64 path: every lattice's populations agree to 1e-10
relative to that lattice's largest population (the FP64 target).  Both
sides evaluate the same formulas in different orders, with different libm
implementations of exp/log; after tens of steps the differences stay at the
1e-14 level, far inside the bound.
"""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import binary_inert, h2_air_synthetic
from oracle import thermo

from helpers import (make_gpu, make_oracle, max_rel_err_per_lattice,
                     oracle_populations, perturbed_box)

pytestmark = pytest.mark.gpu
RTOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


@pytest.mark.parametrize("lattice,shape", [("D3Q27", (6, 5, 4)), ("D2Q9", (7, 5, 1))])
@pytest.mark.parametrize("mechname", ["h2air", "binary"])
def test_init_matches_oracle(lattice, shape, mechname):
    mech = h2_air_synthetic() if mechname == "h2air" else binary_inert()
    w = perturbed_box(shape, lattice, mech=mech)
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o))
    g.close()
    assert np.all(err < 1e-14), err


@pytest.mark.parametrize("lattice,shape,nsteps", [
    ("D3Q27", (10, 7, 5), 12),      # 350 nodes: three blocks and a ragged tail
    ("D2Q9", (23, 17, 1), 15),
])
@pytest.mark.parametrize("chem_lanes,collide_split", [(1, 0), (4, 1), (8, 0)])
def test_perturbed_box_fp64(mech, lattice, shape, nsteps, chem_lanes, collide_split):
    w = perturbed_box(shape, lattice, mech=mech)
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    g.set_launch(chem_lanes, collide_split)
    o.step(nsteps)
    g.step(nsteps)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o))
    mo = o.moments()
    mg = g.moments()
    g.close()
    assert np.all(err < RTOL_FP64), err
    assert np.max(np.abs(mg["T"] - mo["T"].ravel())) < 1e-9 * 1400
    assert np.max(np.abs(mg["Y"] - mo["Y"].reshape(mech.n_species, -1))) < 1e-12


@pytest.mark.parametrize("lattice,shape", [("D3Q27", (9, 4, 3)), ("D2Q9", (16, 6, 1))])
def test_binary_mixture_fp64(lattice, shape):
    mech = binary_inert()
    w = perturbed_box(shape, lattice, mech=mech, T0=300.0, dx=2e-7, amp_Y=0.2, amp_u=5.0)
    w["T_max"] = 600.0
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(20)
    g.step(20)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o))
    g.close()
    assert np.all(err < RTOL_FP64), err


def test_reactor_16cubed_fp64(mech):
    """The homogeneous-reactor workload at its full 16^3 size: element-wise
    parity over the first 10 steps."""
    w = fields.reactor(seed=0)
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(10)
    g.step(10)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o))
    g.close()
    assert np.all(err < RTOL_FP64), err


def test_reactor_full_run_invariants(mech):
    """All 200 steps of the 16^3 reactor, in the launch configuration the
    benchmark times: conservation of mass, momentum, total energy and every
    element (Sec. 3.7, Sec. 3.8), properties that hold at any size."""
    w = fields.reactor(seed=1)
    g = make_gpu(mech, w)
    pops0 = g.populations()
    g.step(w["steps"])
    pops1 = g.populations()
    m1 = g.moments()
    g.close()
    M = mech.n_species
    c = np.array([[(i % 3) - 1, (i // 3) % 3 - 1, i // 9 - 1] for i in range(27)], float)

    def totals(p):
        f, gg = p[M - 1], p[M]
        mass = f.sum()
        mom = c.T @ f.sum(axis=1)
        energy = gg.sum()
        rs = p[: M - 1].sum(axis=1)                     # [M-1, N]
        rs_M = f.sum(axis=0) - rs.sum(axis=0)
        moles = np.concatenate([rs.sum(axis=1), [rs_M.sum()]]) / mech.molar_mass
        return mass, mom, energy, mech.composition.T @ moles
    a0, b0, e0, el0 = totals(pops0)
    a1, b1, e1, el1 = totals(pops1)
    assert abs(a1 - a0) <= 1e-13 * a0
    assert np.all(np.abs(b1 - b0) <= 1e-13 * a0)
    assert abs(e1 - e0) <= 1e-12 * abs(e0)
    assert np.all(np.abs(el1 - el0) <= 1e-12 * el0)
    assert np.all(np.isfinite(m1["T"])) and m1["T"].min() > 1100.0


def test_moments_api_matches_oracle(mech):
    w = perturbed_box((5, 4, 3), "D3Q27", mech=mech)
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(3)
    g.step(3)
    mo, mg = o.moments(), g.moments()
    g.close()
    N = 60
    assert np.allclose(mg["rho"], mo["rho"].ravel(), rtol=1e-13)
    assert np.allclose(mg["u"], mo["u"].reshape(3, N), rtol=1e-10, atol=1e-12)
    assert np.allclose(mg["T"], mo["T"].ravel(), rtol=1e-12)
    assert np.allclose(mg["E"], mo["E"].ravel(), rtol=1e-12)


def test_state_checkpoint_resume_is_bitwise(mech):
    w = perturbed_box((6, 5, 4), "D3Q27", mech=mech)
    a = make_gpu(mech, w)
    a.step(4)
    state = a.get_state()
    a.step(5)
    ref = a.populations()
    b = make_gpu(mech, w)
    b.set_state(state)
    b.step(5)
    got = b.populations()
    a.close()
    b.close()
    assert np.array_equal(got, ref)


def test_device_arrays_through_the_abi(mech):
    """Fields passed as device tensors (on_device = 1) give the same state."""
    torch = pytest.importorskip("torch")
    w = perturbed_box((6, 5, 4), "D3Q27", mech=mech)
    a = make_gpu(mech, w)
    from paper_2108_07605_gb300 import lbm
    b = lbm.Solver(mech, lattice="D3Q27", shape=w["shape"], dx=w["dx"], T_max=w["T_max"])
    dev = [torch.tensor(np.ascontiguousarray(w[k]).reshape(-1), device="cuda",
                        dtype=torch.float64) for k in ("P", "u", "T", "Y")]
    b.init_fields_pressure(*dev)
    a.step(3)
    b.step(3)
    rho = torch.empty(b.N, device="cuda", dtype=torch.float64)
    lbm.lbm_moments(b.h, rho=rho)
    torch.cuda.synchronize()
    assert np.array_equal(a.populations(), b.populations())
    assert np.allclose(rho.cpu().numpy(), a.moments()["rho"], rtol=0, atol=0)
    a.close()
    b.close()


def test_newton_failure_is_reported(mech):
    """A Newton budget of one iteration cannot reach 1e-13: the sticky device
    status surfaces as LBM_ERR_NEWTON at the next synchronising call."""
    from paper_2108_07605_gb300 import lbm
    w = perturbed_box((4, 4, 4), "D3Q27", mech=mech)
    s = lbm.Solver(mech, lattice="D3Q27", shape=w["shape"], dx=w["dx"],
                   T_max=w["T_max"], newton_max_iter=1)
    s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    s.step(1)
    with pytest.raises(lbm.LBMError) as e:
        s.synchronize()
    assert e.value.status == 4
    with pytest.raises(lbm.LBMError):
        s.close()


@pytest.mark.parametrize("case", ["flame", "tube"])
def test_diagnostics_match_the_oracle(mech, case):
    """lbm_diagnostics (one device pass with fixed-order reductions) against
    oracle.diagnostics on the oracle's own state after the same steps."""
    from oracle import diagnostics
    if case == "flame":
        w = fields.flame_1d(nx=48, ny=4, nz=4, x_ign=12, mech=mech)
        nsteps = 15
    else:
        w = fields.microtube(nx=14, ny=10, nz=10, radius=4.5, mech=mech)
        nsteps = 8
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(nsteps)
    g.step(nsteps)
    mo = o.moments()
    fluid = None if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
    ref = diagnostics.diagnostics(mech, mo["rho"], mo["u"], mo["T"], mo["Y"], w["dx"], 3,
                                  w["shape"][0], fluid)
    got = g.diagnostics()
    g.close()
    assert abs(ref["hrr_integral"]) > 0.0
    for k in ("hrr_integral", "hrr_max", "T_max", "u_max"):
        assert got[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-12), k
    assert got["flame_x"] == pytest.approx(ref["flame_x"], abs=1e-12)


@pytest.mark.parametrize("collide_split", [0, 1])
def test_wilke_viscosity_option(collide_split):
    """The Wilke mixing-rule viscosity option, element-wise against the
    oracle with the same option (FP64, 1e-10), in both collision kernels."""
    from lbm_workloads.mechanism import with_viscosity_model
    mech = with_viscosity_model(h2_air_synthetic(), "wilke")
    w = perturbed_box((9, 6, 5), "D3Q27", mech=mech)
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    g.set_launch(-1, collide_split)
    o.step(10)
    g.step(10)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o))
    g.close()
    assert np.all(err < RTOL_FP64), err
