"""GPU parity on the paths the full-size runs take, over longer horizons:

* the reaction sub-step counts l = 1 and l = 4 (Sec. 2.4, Eq. R3) beside the
  default l = 2, on a periodic box and on the flame layout (inlet + LODI
  outlet; the interface nodes' sub-steps run in their own kernel);
* the 16^3 reactor over all 200 of its steps and the 1024x4x4 flame over 50,
  element-wise;
* a 100x40x40 segment of the microtube (the staircase circular wall of the
  600x40x40 tube with its TMS temperature ramp, inlet and outlet) over 30
  steps: FP64 element-wise, FP32 storage (float-float and FP64 chemistry)
  and FP16 offsets held to their stated field tolerances.

FP64 bound: every population within 1e-10 of the oracle relative to its
lattice's largest population, and, element by element, within
1e-10 |ref| + 1e-13 max|lattice| (the absolute floor covers populations
that are near zero).  Mixed-precision tolerances are those of
test_gpu_mixed.py."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, make_oracle, max_rel_err_per_lattice, oracle_populations

pytestmark = pytest.mark.gpu
RTOL_FP64 = 1e-10
FLOOR = 1e-13
TOL = {"fp32": dict(Y=2e-5, T=0.05, u=5e-3, rho=1e-4),
       "fp32c64": dict(Y=2e-5, T=0.05, u=5e-3, rho=1e-4),
       "fp16": dict(Y=1e-3, T=5.0, u=3.0, rho=3e-2)}


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def elementwise_ok(got, ref, mask=None):
    """|got - ref| <= 1e-10 |ref| + 1e-13 max|lattice| for every element;
    returns (ok, worst ratio of |got - ref| to that bound)."""
    if mask is not None:
        got, ref = got[:, :, mask], ref[:, :, mask]
    scale = np.max(np.abs(ref), axis=(1, 2), keepdims=True)
    bound = RTOL_FP64 * np.abs(ref) + FLOOR * scale
    ratio = np.abs(got - ref) / bound
    return bool(np.all(ratio <= 1.0)), float(ratio.max())


def _fp64_parity(mech, w, nsteps, substeps=None):
    if substeps:
        w["substeps"] = substeps
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(nsteps)
    g.step(nsteps)
    mask = None if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
    got, ref = g.populations(), oracle_populations(o)
    g.close()
    lat = max_rel_err_per_lattice(got, ref, mask)
    ok, worst = elementwise_ok(got, ref, mask)
    return lat, ok, worst


@pytest.mark.parametrize("substeps", [1, 4])
@pytest.mark.parametrize("case", ["box", "flame"])
def test_substep_counts(mech, case, substeps):
    if case == "box":
        w = fields.perturbed_box((10, 7, 5), "D3Q27", mech=mech)
    else:
        w = fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10)
    lat, ok, worst = _fp64_parity(mech, w, 12, substeps)
    assert np.all(lat < RTOL_FP64), lat
    assert ok, worst


def test_reactor_all_200_steps_elementwise(mech):
    w = fields.reactor(seed=0)
    lat, ok, worst = _fp64_parity(mech, w, w["steps"])
    assert np.all(lat < RTOL_FP64), lat
    assert ok, worst


def test_full_flame_50_steps_elementwise(mech):
    w = fields.flame_1d()
    lat, ok, worst = _fp64_parity(mech, w, 50)
    assert np.all(lat < RTOL_FP64), lat
    assert ok, worst


TUBE_STEPS = 30


@pytest.fixture(scope="module")
def tube_oracle(mech):
    """The oracle on the 100x40x40 tube segment after TUBE_STEPS steps."""
    w = fields.microtube(nx=100, mech=mech)
    o = make_oracle(mech, w)
    o.step(TUBE_STEPS)
    return w, oracle_populations(o).copy(), o.moments()


def test_tube_segment_fp64_elementwise(mech, tube_oracle):
    w, ref, _ = tube_oracle
    g = make_gpu(mech, w)
    g.step(TUBE_STEPS)
    got = g.populations()
    g.close()
    mask = ~np.asarray(w["solid"]).reshape(-1)
    lat = max_rel_err_per_lattice(got, ref, mask)
    ok, worst = elementwise_ok(got, ref, mask)
    assert np.all(lat < RTOL_FP64), lat
    assert ok, worst


@pytest.mark.parametrize("precision", ["fp32", "fp32c64", "fp16"])
def test_tube_segment_reduced_precision_fields(mech, tube_oracle, precision):
    w, _, mo = tube_oracle
    g = make_gpu(mech, w, precision=precision)
    g.step(TUBE_STEPS)
    mg = g.moments()
    g.close()
    keep = ~np.asarray(w["solid"]).reshape(-1)
    M = mech.n_species
    tol = TOL[precision]
    dY = np.abs(mg["Y"] - mo["Y"].reshape(M, -1))[:, keep].max()
    dT = np.abs(mg["T"] - mo["T"].ravel())[keep].max()
    du = np.abs(mg["u"] - mo["u"].reshape(3, -1))[:, keep].max()
    drho = (np.abs(mg["rho"] - mo["rho"].ravel()) / mo["rho"].ravel())[keep].max()
    assert dY <= tol["Y"], dY
    assert dT <= tol["T"], dT
    assert du <= tol["u"], du
    assert drho <= tol["rho"], drho


def test_substeps_converge_to_radau_on_the_gpu(mech):
    """The GPU's reaction sub-steps (Sec. 2.4 Eq. R3, the discussion after
    it): a uniform, still 4^3 periodic box is a constant-U reactor whose
    species advance only by the l explicit sub-steps per step.  Against a
    tight-tolerance Radau solution of the same reactor over the same time,
    the OH density's error falls at first order in dt/l: l = 2 and l = 4
    halve it and quarter it (within 1.6-2.5 per doubling), and stays small."""
    scipy = pytest.importorskip("scipy.integrate")
    from oracle import chemistry, thermo
    w = fields.reactor(n=4, T0=1300.0, perturbation=0.0, dx=12.5e-6, mech=mech)
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"]).reshape(-1)[0]
    Y0 = np.asarray(w["Y"]).reshape(mech.n_species, -1)[:, 0]
    T0 = 1300.0
    U = float(thermo.mixture_U(mech, Y0[:, None], np.array([T0]))[0])
    r0 = rho * Y0
    iOH = mech.index("OH")
    errs = []
    for l in (1, 2, 4):
        w["substeps"] = l
        g = make_gpu(mech, w)
        dt = g.info.dt
        nsteps = int(round(1.0e-5 / dt))
        g.step(nsteps)
        m = g.moments()
        g.close()
        r_gpu = m["rho"][0] * m["Y"][:, 0]
        t_end = nsteps * dt

        def rhs(t, r):
            T = thermo.temperature_from_energy(mech, (r / rho)[:, None], np.array([U]),
                                               np.array([rhs.T]))
            rhs.T = T[0]
            return chemistry.production_rates(mech, T, r[:, None])[:, 0]
        rhs.T = T0
        ref = scipy.solve_ivp(rhs, (0.0, t_end), r0, method="Radau", rtol=1e-12,
                              atol=1e-18).y[:, -1]
        assert abs(ref[iOH] - r0[iOH]) > 10 * abs(r0[iOH]) + 1e-12   # OH has grown
        errs.append(abs(r_gpu[iOH] - ref[iOH]) / abs(ref[iOH]))
    assert errs[0] < 1e-2, errs
    for a, b in zip(errs, errs[1:]):
        assert 1.6 < a / b < 2.5, errs
