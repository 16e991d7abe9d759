"""The FP32-storage path (populations, moments, gradients, diffusion-velocity
solve and collision in FP32; temperature Newton, transport and chemistry in
FP64) against the FP64 oracle, per field, after tens of steps.

Stated tolerances (max over nodes, fluid nodes only), measured margins about
4x: mass fractions |dY| <= 2e-5, temperature |dT| <= 0.05 K, velocity
|du| <= 5e-3 m/s, density |drho|/rho <= 1e-4.  They come from FP32 rounding
of the stored populations (relative 6e-8 per population) accumulated over
the steps; they are not parity bounds of the FP64 kind."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import make_gpu, make_oracle

pytestmark = pytest.mark.gpu
TOL = dict(Y=2e-5, T=0.05, u=5e-3, rho=1e-4)


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


CASES = {
    "periodic box": (lambda m: fields.perturbed_box((10, 7, 5), "D3Q27", mech=m), 12),
    "flame layout": (lambda m: fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10), 50),
    "channel layout": (lambda m: fields.channel_2d(nx=30, ny=9), 50),
    "tube layout": (lambda m: fields.microtube(nx=10, ny=9, nz=9, radius=3.6), 30),
    "flame 1024x4x4": (lambda m: fields.flame_1d(), 20),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp32_storage_field_errors(mech, case):
    make, nsteps = CASES[case]
    w = make(mech)
    o = make_oracle(mech, w)
    o.step(nsteps)
    mo = o.moments()
    g = make_gpu(mech, w, precision="fp32")
    g.step(nsteps)
    mg = g.moments()
    g.close()
    keep = np.ones(g.N, bool) if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
    M, D = mech.n_species, o.vs.dim
    dY = np.abs(mg["Y"] - mo["Y"].reshape(M, -1))[:, keep].max()
    dT = np.abs(mg["T"] - mo["T"].ravel())[keep].max()
    du = np.abs(mg["u"][:D] - mo["u"].reshape(D, -1))[:, keep].max()
    drho = (np.abs(mg["rho"] - mo["rho"].ravel()) / mo["rho"].ravel())[keep].max()
    assert dY <= TOL["Y"], dY
    assert dT <= TOL["T"], dT
    assert du <= TOL["u"], du
    assert drho <= TOL["rho"], drho
