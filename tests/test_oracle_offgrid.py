"""Pins of the oracle's off-grid TMS targets (Sec. 4.2.2, last paragraph;
reading R20: linear interpolation along the wall normal between the wall and
the fluid neighbour most aligned with it).

* Decay of the slowest mode of a circular pipe (a single-fluid binary
  mixture at rest but for u_x = U0 J0(2.4048 r / R), periodic along the
  axis, isothermal TMS walls at r = R): the NS rate is nu (2.4048 / R)^2.
  With the staircase reading (targets at the interface node) the rate error
  falls at first order in 1/R; with the interpolated targets it is several
  times smaller at every radius and falls faster.
* With a zero wall distance everywhere the interpolated targets are the
  wall values, so the step equals the staircase step exactly.
"""
import numpy as np
from scipy.special import j0

from lbm_workloads import fields
from lbm_workloads.mechanism import P_STANDARD, R_UNIVERSAL, binary_inert, h2_air_synthetic
from oracle import OracleLBM, thermo
from oracle.transport import relaxation

from helpers import make_oracle

J0_ZERO = 2.404825557695773


def pipe_decay_error(radius, offgrid, nu_lat=0.05, theta0=0.2, every=10, T0=300.0):
    """(measured / NS decay rate - 1) of the slowest pipe mode."""
    mech = binary_inert()
    R = R_UNIVERSAL / mech.molar_mass[0]
    c = np.sqrt(R * T0 / theta0)
    rho0 = P_STANDARD / (R * T0)
    mu = mech.mu0 * (T0 / 298.15) ** mech.mu_T_exponent
    dx = mu / rho0 / (c * nu_lat)
    n = int(np.ceil(2 * radius)) + 3
    solid, dist, normal = fields.pipe_wall_geometry(n, n, radius)
    g = (n, n, 1)
    spec = dict(faces=("periodic",) * 6, solid=solid[:, :, None], solid_kind="tms",
                wall_T=np.full(g, T0))
    if offgrid:
        spec["wall_dist"] = dist[:, :, None]
        spec["wall_normal"] = normal[:, :, :, None]
    o = OracleLBM(mech, "D3Q27", (1, n, n), dx, c_ref=c, substeps=1, boundaries=spec)
    r = radius - dist
    u = np.zeros((3,) + g)
    u[0] = (1e-3 * c * np.where(r < radius, j0(J0_ZERO * np.minimum(r, radius) / radius),
                                0.0))[:, :, None]
    Y = np.stack([np.full(g, 0.5), np.full(g, 0.5)])
    T = np.full(g, T0)
    o.init_fields(thermo.density_from_pressure(mech, np.full(g, P_STANDARD), T, Y), u, T, Y)
    rel = relaxation(mech, o.units, np.full(g, rho0), Y, T)
    nu = (1.0 / rel["omega"].ravel()[0] - 0.5) * theta0
    exact = nu * (J0_ZERO / radius) ** 2
    nsteps = int(1.0 / exact)
    fluid = ~solid[:, :, None]
    ts, logs = [], []
    for s in range(0, nsteps + 1, every):
        if s:
            o.step(every)
        ts.append(s)
        logs.append(np.log(np.sum(o.moments()["u"][0][fluid])))
    ts, logs = np.array(ts, float)[len(ts) // 3:], np.array(logs)[len(ts) // 3:]
    A = np.vstack([ts, np.ones_like(ts)]).T
    return -np.linalg.lstsq(A, logs, rcond=None)[0][0] / exact - 1.0


def test_interpolated_targets_converge_faster_than_the_staircase():
    stair = [pipe_decay_error(R, False) for R in (4.5, 6.5)]
    inter = [pipe_decay_error(R, True) for R in (4.5, 6.5, 9.5)]
    # staircase: first order (error ratio ~ R ratio)
    assert stair[0] / stair[1] < 1.7
    for s, i in zip(stair, inter):
        assert abs(i) < abs(s) / 3.0
    # interpolated: faster than first order over 4.5 -> 9.5 (ratio 2.1 of R)
    assert abs(inter[0]) / abs(inter[2]) > 2.1 ** 1.4
    assert abs(inter[2]) < 0.06


def test_zero_wall_distance_is_the_staircase_step():
    mech = h2_air_synthetic()
    w = fields.microtube(nx=6, ny=9, nz=9, radius=3.6, mech=mech, offgrid=True)
    w["wall_dist"] = np.zeros_like(w["wall_dist"])
    a = make_oracle(mech, w)
    w2 = {k: v for k, v in w.items() if k not in ("wall_dist", "wall_normal")}
    b = make_oracle(mech, w2)
    a.step(3)
    b.step(3)
    fluid = ~w["solid"]
    assert np.array_equal(a.pops[:, :, fluid], b.pops[:, :, fluid])
