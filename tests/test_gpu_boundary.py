"""GPU parity of the boundary conditions (Sec. 4) against the oracle:
bounce-back box, flux inlet + LODI outlet (flame layout), Tamm-Mott-Smith
walls with a temperature ramp and a parabolic inlet (channel layout, D2Q9),
staircase solid walls (microtube layout) with targets at the interface node
or interpolated off the grid along the wall normal, and the full-size
1024x4x4 flame in the launch configuration the benchmark times.  FP64 tolerance: 1e-10
relative per lattice, as for the periodic tests; solid nodes are excluded
(their populations are not defined)."""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import h2_air_synthetic

from helpers import (make_gpu, make_oracle, max_rel_err_per_lattice,
                     oracle_populations)

pytestmark = pytest.mark.gpu
RTOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _compare(mech, w, nsteps):
    o = make_oracle(mech, w)
    g = make_gpu(mech, w)
    o.step(nsteps)
    g.step(nsteps)
    mask = None if w.get("solid") is None else ~np.asarray(w["solid"]).reshape(-1)
    err = max_rel_err_per_lattice(g.populations(), oracle_populations(o), mask)
    g.close()
    return err


def test_bounce_back_box(mech):
    w = fields.perturbed_box((6, 5, 4), "D3Q27", mech=mech, amp_u=2.0, T0=900.0, dx=2e-5)
    w["faces"] = ("bounce_back",) * 6
    err = _compare(mech, w, 8)
    assert np.all(err < RTOL_FP64), err


def test_flame_layout_inlet_outlet(mech):
    w = fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10)
    err = _compare(mech, w, 12)
    assert np.all(err < RTOL_FP64), err


@pytest.mark.parametrize("precision", ["fp64"])
def test_channel_layout_tms_walls_parabolic_inlet(mech, precision):
    w = fields.channel_2d(nx=30, ny=9, dx=25e-6)
    err = _compare(mech, w, 10)
    assert np.all(err < RTOL_FP64), err


def test_tube_layout_staircase_walls(mech):
    w = fields.microtube(nx=10, ny=9, nz=9, radius=3.6, dx=25e-6)
    err = _compare(mech, w, 6)
    assert np.all(err < RTOL_FP64), err


def test_full_flame_first_steps(mech):
    """The 1024x4x4 flame at full size, element-wise over the first steps."""
    w = fields.flame_1d()
    err = _compare(mech, w, 3)
    assert np.all(err < RTOL_FP64), err


def test_flame_layout_simplified_inlet(mech):
    """The simplified flux inlet (Sec. 4.3, last paragraph) on the flame
    layout: populations against the oracle with the same option."""
    w = fields.flame_1d(nx=40, ny=3, nz=2, x_ign=10)
    w["inlet"] = dict(w["inlet"], simplified=True)
    err = _compare(mech, w, 12)
    assert np.all(err < RTOL_FP64), err


@pytest.mark.parametrize("shape,radius,nsteps", [((10, 9, 9), 3.6, 6), ((20, 40, 40), 19.0, 5)])
def test_tube_offgrid_targets(mech, shape, radius, nsteps):
    """Off-grid TMS targets (Sec. 4.2.2, last paragraph): the circular wall
    given by its normal distance and normal per node, targets interpolated
    towards the fluid, against the oracle with the same geometry."""
    nx, ny, nz = shape
    w = fields.microtube(nx=nx, ny=ny, nz=nz, radius=radius, dx=25e-6, offgrid=True)
    err = _compare(mech, w, nsteps)
    assert np.all(err < RTOL_FP64), err
