"""The reduced-precision paths against the FP64 oracle, per field, after tens
of steps.

FP32 storage (populations, moments, gradients, transport, diffusion-velocity
solve and collision in FP32; temperature Newton and chemistry in
float-float).  Stated tolerances (max over fluid nodes), measured margins
3-4x: mass fractions |dY| <= 2e-5, temperature |dT| <= 0.05 K, velocity
|du| <= 5e-3 m/s, density |drho|/rho <= 1e-4.  They come from FP32 rounding
of the stored populations (relative 6e-8 per population) accumulated over
the steps; they are not parity bounds of the FP64 kind.

FP32 storage with native FP64 chemistry (chem_fp64: the temperature
Newton solves and the reaction sub-steps in FP64, everything else as the
FP32 path): the same stated tolerances, which come from the FP32 storage.

FP16 offset storage (the FP32 path's arithmetic, populations stored as FP16
offsets from the mean initial equilibrium with per-lattice scales): each
stored deviation keeps 11 significant bits, and in this low-Mach flow
(|u| ~ 1e-3 of the lattice speed) the velocity moment is a small difference
of quantised populations.  Stated tolerances, measured margins about 3x:
|dY| <= 1e-3, |dT| <= 5 K, |du| <= 3 m/s, |drho|/rho <= 3e-2 (measured
maxima 3.2e-4, 1.5 K, 1.0 m/s, 1.1e-2 on the flame layout)."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, make_oracle

pytestmark = pytest.mark.gpu
TOL = {"fp32": dict(Y=2e-5, T=0.05, u=5e-3, rho=1e-4),
       "fp32c64": dict(Y=2e-5, T=0.05, u=5e-3, rho=1e-4),
       "fp16": dict(Y=1e-3, T=5.0, u=3.0, rho=3e-2)}


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


CASES = {
    "periodic box": (lambda m: fields.perturbed_box((10, 7, 5), "D3Q27", mech=m), 12),
    "flame layout": (lambda m: fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10), 50),
    "channel layout": (lambda m: fields.channel_2d(nx=30, ny=9), 50),
    "tube layout": (lambda m: fields.microtube(nx=10, ny=9, nz=9, radius=3.6), 30),
    "tube layout, off-grid targets": (
        lambda m: fields.microtube(nx=10, ny=9, nz=9, radius=3.6, offgrid=True), 30),
    "flame 1024x4x4": (lambda m: fields.flame_1d(), 20),
}


@pytest.mark.parametrize("precision", ["fp32", "fp32c64", "fp16"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_reduced_precision_field_errors(mech, case, precision):
    make, nsteps = CASES[case]
    w = make(mech)
    o = make_oracle(mech, w)
    o.step(nsteps)
    mo = o.moments()
    tol = TOL[precision]
    g = make_gpu(mech, w, precision=precision)
    g.step(nsteps)
    mg = g.moments()
    g.close()
    keep = np.ones(g.N, bool) if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
    M, D = mech.n_species, o.vs.dim
    dY = np.abs(mg["Y"] - mo["Y"].reshape(M, -1))[:, keep].max()
    dT = np.abs(mg["T"] - mo["T"].ravel())[keep].max()
    du = np.abs(mg["u"][:D] - mo["u"].reshape(D, -1))[:, keep].max()
    drho = (np.abs(mg["rho"] - mo["rho"].ravel()) / mo["rho"].ravel())[keep].max()
    assert dY <= tol["Y"], dY
    assert dT <= tol["T"], dT
    assert du <= tol["u"], du
    assert drho <= tol["rho"], drho


def test_fp16_checkpoint_carries_the_codec(mech):
    """An FP16 checkpoint restores into a handle whose own codec came from
    other initial fields: the solve continues bit for bit."""
    w = fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10)
    a = make_gpu(mech, w, precision="fp16")
    a.step(5)
    state = a.get_state()
    a.step(5)
    w2 = fields.perturbed_box((40, 3, 2), "D3Q27", mech=mech)
    w2.update({k: w[k] for k in ("faces", "inlet", "outlet", "lattice", "shape", "dx",
                                 "T_max", "substeps") if k in w})
    b = make_gpu(mech, w2, precision="fp16")
    b.set_state(state)
    b.step(5)
    assert np.array_equal(a.populations(), b.populations())
    a.close()
    b.close()
