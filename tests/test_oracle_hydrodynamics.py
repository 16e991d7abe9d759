"""Hydrodynamic pins of the oracle's momentum and energy lattices against the
Navier-Stokes-Fourier limit the paper states (Sec. 3.5, Eqs. dtrho-lambda,
qneq), on small periodic or walled boxes of a single-fluid binary mixture.
Each pin ties a part of the collision that the conservation and moment pins
cannot see to a closed form; the planted-mistake tests below show that a
wrong sign or factor there makes the pin fail.

* Sound (Eqs. dtu, dtE with NSmix, mu, varsigma, qneq, lambda): a linear
  acoustic wave travels at sqrt(gamma theta) + U0 and decays at
  Gamma = k^2/2 [2 nu (1 - 1/D) + varsigma/rho + (gamma - 1) alpha], with
  nu = (1/omega - 1/2) theta, varsigma/rho = (1/omega - 1/2)(2/D - R/C_v)
  theta and alpha = (1/omega_1 - 1/2) theta.  At theta = 0.2 the lattice's
  missing third moment is large, so the rate depends on the extended
  equilibrium (Eq. Pex); a background velocity U0 along the wave vector
  (Galilean invariance, the extension's purpose, Sec. 3.3) must leave the
  rate unchanged, which needs the energy terms q^ex (Eq. qex) and
  u.(P - P^eq) (Eq. gstareq1mom).  A shear wave cannot pin the extension:
  its divergence-free flow gives d_alpha Phi_alpha = 0.
* Conduction (Eq. lambda): an isobaric temperature mode decays at alpha k^2,
  with and without a background flow; steady conduction between two TMS
  walls (Sec. 4.2.2) gives a profile whose Kirchhoff variable int lambda dT
  (here T^(1 + 0.7), lambda ~ T^0.7) is linear between the walls, with a
  wall temperature jump that falls at first order under refinement.
* Interdiffusion energy flux (Eq. qneq, second term; Eqs. qdiff,
  corrFourier): two species of equal molar mass but different formation
  enthalpies interdiffuse at uniform temperature and pressure.  The exact
  energy equation then keeps T uniform (the enthalpy flux rho sum H_a Y_a
  V_a is exactly the enthalpy the species carry), while a wrong q^diff or
  q^corr moves T by a fraction of the enthalpy jump over c_p.
* Reading R5 (Eq. momentum1): a near-zero species density with mixed-sign
  populations and |j_a| >= rho_a takes u_a = u, which keeps its populations
  bounded at a TMS wall node; without that branch they grow by orders of
  magnitude.
"""
import numpy as np
import pytest

from lbm_workloads.mechanism import P_STANDARD, R_UNIVERSAL, binary_inert, h2_air_synthetic
from oracle import OracleLBM, thermo
from oracle.transport import relaxation

from oracle_mutations import mutation

THETA0 = 0.2          # lattice temperature R T / c^2 (far from the D3Q27 value 1/3)
NU_LAT = 0.03         # lattice kinematic viscosity
GAMMA = 1.4           # c_p / c_v of the binary table (c_p = 3.5 R)
R_OVER_CV = 1.0 / 2.5


def _single_fluid(T0, nu_lat=NU_LAT, theta0=THETA0, mech=None):
    """(mech, R, c, dx) so that theta = theta0 and nu_lat hold at T0, P0."""
    mech = mech or binary_inert()
    R = R_UNIVERSAL / mech.molar_mass[0]
    c = np.sqrt(R * T0 / theta0)
    rho0 = P_STANDARD / (R * T0)
    mu = mech.mu0 * (T0 / 298.15) ** mech.mu_T_exponent
    dx = mu / rho0 / (c * nu_lat)
    return mech, R, c, dx


def _fit_rate(ts, values):
    A = np.vstack([ts, np.ones_like(ts)]).T
    return -np.linalg.lstsq(A, values, rcond=None)[0][0]


def acoustic_wave(U0_frac, nx=32, nsteps=400, every=5, eps=1e-4, oracle_cls=OracleLBM):
    """Right-running linear acoustic wave on a background U0 = U0_frac
    sqrt(theta).  Returns (measured/predicted decay rate, measured/predicted
    phase speed)."""
    T0 = 300.0
    mech, R, c, dx = _single_fluid(T0)
    cs = np.sqrt(GAMMA * THETA0)
    U0 = U0_frac * np.sqrt(THETA0)
    x = np.arange(nx)
    k = 2 * np.pi / nx
    g = (1, 1, nx)
    wave = np.cos(k * x)[None, None, :] * np.ones(g)
    P = P_STANDARD * (1 + GAMMA * eps * wave)            # isentropic relations
    T = T0 * (1 + (GAMMA - 1) * eps * wave)
    u = np.zeros((3,) + g)
    u[0] = (U0 + cs * eps * wave) * c
    Y = np.stack([np.full(g, 0.5), np.full(g, 0.5)])
    o = oracle_cls(mech, "D3Q27", (nx, 1, 1), dx, c_ref=c, substeps=1)
    o.init_fields(thermo.density_from_pressure(mech, P, T, Y), u, T, Y)
    rho0 = P_STANDARD / (R * T0)
    rel = relaxation(mech, o.units, np.full(g, rho0), Y, np.full(g, T0))
    om, om1 = rel["omega"].ravel()[0], rel["omega1"].ravel()[0]
    nu = (1 / om - 0.5) * THETA0
    alpha = (1 / om1 - 0.5) * THETA0
    D = 3
    zeta = (1 / om - 0.5) * (2.0 / D - R_OVER_CV) * THETA0
    gamma_pred = 0.5 * k * k * (2 * nu * (1 - 1.0 / D) + zeta + (GAMMA - 1) * alpha)
    ts, logamp, phase = [], [], []
    for s in range(0, nsteps + 1, every):
        if s:
            o.step(every)
        rk = np.sum(o.moments_of(o.pops)["rho"][0, 0] * np.exp(-1j * k * x)) * 2 / nx
        ts.append(s)
        logamp.append(np.log(abs(rk)))
        phase.append(np.angle(rk))
    ts = np.array(ts, dtype=float)
    rate = _fit_rate(ts, np.array(logamp))
    speed = _fit_rate(ts, np.unwrap(np.array(phase))) / k
    return rate / gamma_pred, speed / (U0 + cs)


def thermal_mode(U0_frac, nx=32, nsteps=600, every=10, eps=1e-3, oracle_cls=OracleLBM):
    """Isobaric temperature mode T = T0 (1 + eps sin kx) at rest or on a
    background flow.  Returns measured decay rate / (alpha k^2)."""
    T0 = 300.0
    mech, R, c, dx = _single_fluid(T0)
    x = np.arange(nx)
    k = 2 * np.pi / nx
    g = (1, 1, nx)
    P = np.full(g, P_STANDARD)
    T = T0 * (1 + eps * np.sin(k * x))[None, None, :] * np.ones(g)
    u = np.zeros((3,) + g)
    u[0] = U0_frac * np.sqrt(THETA0) * c
    Y = np.stack([np.full(g, 0.5), np.full(g, 0.5)])
    o = oracle_cls(mech, "D3Q27", (nx, 1, 1), dx, c_ref=c, substeps=1)
    o.init_fields(thermo.density_from_pressure(mech, P, T, Y), u, T, Y)
    rho0 = P_STANDARD / (R * T0)
    rel = relaxation(mech, o.units, np.full(g, rho0), Y, np.full(g, T0))
    alpha = (1 / rel["omega1"].ravel()[0] - 0.5) * THETA0
    ts, logamp = [], []
    for s in range(0, nsteps + 1, every):
        if s:
            o.step(every)
        ts.append(s)
        logamp.append(np.log(abs(np.sum(o.T[0, 0] * np.exp(-1j * k * x)) * 2 / nx)))
    return _fit_rate(np.array(ts, dtype=float), np.array(logamp)) / (alpha * k * k)


def interdiffusion_T_drift(nx=32, nsteps=200, dY=0.2, dh=1.0e4, oracle_cls=OracleLBM):
    """Binary interdiffusion at uniform T and P between species whose
    formation enthalpies differ by dh (J/mol).  Returns the largest |T - T0|
    over the run divided by the scale dh/(m c_p) dY."""
    T0 = 300.0
    mech, R, c, dx = _single_fluid(T0, mech=binary_inert(h_formation=(0.0, dh)))
    x = np.arange(nx)
    k = 2 * np.pi / nx
    g = (1, 1, nx)
    YA = (0.5 + dY * np.sin(k * x))[None, None, :] * np.ones(g)
    Y = np.stack([YA, 1 - YA])
    P, T, u = np.full(g, P_STANDARD), np.full(g, T0), np.zeros((3,) + g)
    o = oracle_cls(mech, "D3Q27", (nx, 1, 1), dx, c_ref=c, substeps=1)
    o.init_fields(thermo.density_from_pressure(mech, P, T, Y), u, T, Y)
    scale = dh / mech.molar_mass[0] / (3.5 * R) * dY
    drift = 0.0
    for _ in range(nsteps // 20):
        o.step(20)
        drift = max(drift, float(np.max(np.abs(o.moments()["T"] - T0))))
    # the mixture did interdiffuse
    Yk = abs(np.sum(o.moments()["Y"][0, 0, 0] * np.exp(-1j * k * x)) * 2 / nx)
    assert Yk < 0.9 * dY
    return drift / scale


def tms_conduction(ny, nsteps, T1=300.0, T2=330.0, nu_lat=0.1, oracle_cls=OracleLBM):
    """Steady conduction between TMS walls at T1 (y = 0) and T2 (y = ny-1),
    D2Q9, started from the exact constant-flux profile.  Returns (largest
    second difference of the Kirchhoff variable over the interior nodes,
    relative; wall temperature jumps at the first interior nodes, K)."""
    Tm = 0.5 * (T1 + T2)
    mech, R, c, dx = _single_fluid(Tm, nu_lat=nu_lat)
    e = 1.0 + mech.mu_T_exponent             # lambda ~ mu ~ T^0.7: int lambda dT ~ T^e
    y = np.arange(ny) / (ny - 1)
    exact = (T1 ** e + (T2 ** e - T1 ** e) * y) ** (1 / e)
    g = (1, ny, 1)
    wall = np.broadcast_to(exact[None, :, None], g).copy()
    spec = dict(faces=("periodic", "periodic", "tms", "tms", "periodic", "periodic"),
                wall_T=wall)
    o = oracle_cls(mech, "D2Q9", (1, ny, 1), dx, c_ref=c, substeps=1, boundaries=spec)
    Y = np.stack([np.full(g, 0.5), np.full(g, 0.5)])
    o.init_fields(thermo.density_from_pressure(mech, np.full(g, P_STANDARD), wall, Y),
                  np.zeros((3,) + g), wall, Y)
    o.step(nsteps)
    m = o.moments()
    Ty = m["T"][0, :, 0]
    assert abs(Ty[0] - T1) < 1e-9 and abs(Ty[-1] - T2) < 1e-9     # TMS targets
    assert np.max(np.abs(m["u"])) < 1e-4              # at rest (m/s; c = 667 m/s)
    K = Ty[1:-1] ** e
    d2 = np.max(np.abs(K[2:] - 2 * K[1:-1] + K[:-2])) / np.mean(K)
    return d2, (Ty[1] - exact[1], Ty[-2] - exact[-2])


# ---------------------------------------------------------------- pins
def test_acoustic_wave_speed_attenuation_and_galilean_invariance():
    r0, s0 = acoustic_wave(0.0)
    r2, s2 = acoustic_wave(0.2)
    assert abs(s0 - 1) < 3e-3 and abs(s2 - 1) < 3e-3        # sqrt(gamma theta) (+ U0)
    assert abs(r0 - 1) < 0.03 and abs(r2 - 1) < 0.03         # NS attenuation
    assert abs(r2 / r0 - 1) < 6e-3                           # unchanged by U0


@pytest.mark.parametrize("U0_frac", [0.0, 0.2])
def test_thermal_mode_decays_at_alpha_k2(U0_frac):
    assert abs(thermal_mode(U0_frac) - 1) < 0.015


def test_interdiffusion_of_different_enthalpies_keeps_T_uniform():
    coarse = interdiffusion_T_drift(nx=32, nsteps=200)
    fine = interdiffusion_T_drift(nx=64, nsteps=800)
    assert coarse < 5e-3
    assert coarse / fine > 3.0                                # second order


def test_tms_walls_conduct_with_a_linear_kirchhoff_profile():
    d2_12, jump_12 = tms_conduction(12, 1000)
    d2_24, jump_24 = tms_conduction(24, 2000)
    assert d2_12 < 1e-7 and d2_24 < 1e-7
    assert max(abs(j) for j in jump_12) < 0.01 * 30.0
    assert all(a / b > 1.6 for a, b in zip(jump_12, jump_24))   # first order


def _r5_growth():
    """A 3x4x3 box of the H2/air table at rest at 300 K (chemistry frozen)
    between TMS walls on the y faces; the H-atom lattice is replaced by a
    near-zero density (1e-12 of rho) whose +x/-x populations carry
    |j_x| = 1000 rho_a, of mixed signs.  The TMS step forms the local
    equilibrium at each species' own velocity (Sec. 4.2.2, step 3), where
    j_a / rho_a = 1000 would enter a product form of degree two per axis.
    Returns max |f_H| / rho_a after one step."""
    mech = h2_air_synthetic()
    from lbm_workloads import fields
    w = fields.perturbed_box((3, 4, 3), "D3Q27", mech=mech, amp_u=0.0, seed=4, T0=300.0)
    spec = dict(faces=("periodic", "periodic", "tms", "tms", "periodic", "periodic"),
                wall_T=300.0)
    o = OracleLBM(mech, "D3Q27", (3, 4, 3), 2e-5, T_max=3000.0, substeps=2, boundaries=spec)
    o.init_fields(thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"]), w["u"], w["T"],
                  w["Y"])
    a = mech.index("H")
    rho_a = 1e-12 * o.pops[mech.n_species - 1].sum(axis=0)
    o.pops[a] = rho_a * o.pops[a] / o.pops[a].sum(axis=0)
    ip, im = o.vs._index((1, 0, 0)), o.vs._index((-1, 0, 0))
    o.pops[a, ip] += 500.0 * rho_a
    o.pops[a, im] -= 500.0 * rho_a
    m0 = o.moments_of(o.pops)
    assert np.all(np.abs(m0["j_s"][a][0]) >= m0["rho_s"][a])      # the branch's condition
    o.step(1)
    return float(np.max(np.abs(o.pops[a]) / rho_a))


def test_r5_branch_keeps_a_near_zero_species_bounded():
    from oracle.lbm import species_velocity_undefined
    # never taken for non-negative populations with a positive density
    rng = np.random.default_rng(2)
    pops = rng.uniform(0.0, 1.0, size=(27, 50))
    c = OracleLBM(h2_air_synthetic(), "D3Q27", (1, 1, 1), 1e-5).vs.c.astype(float)
    assert not np.any(species_velocity_undefined(pops.sum(axis=0), c.T @ pops))
    assert _r5_growth() < 1000.0          # no larger than the planted populations (500)


# ------------------------------------------------ planted mistakes fail the pins
@pytest.mark.parametrize("name", ["Pex_dropped", "Pex_half", "qex_sign", "qex_dropped",
                                  "uP_sign", "uP_dropped"])
def test_acoustic_pin_catches(name):
    mod = mutation(name)
    try:
        r0, _ = acoustic_wave(0.0, oracle_cls=mod.OracleLBM)
        r2, _ = acoustic_wave(0.2, oracle_cls=mod.OracleLBM)
    except thermo.NewtonError:
        return                                  # went unstable: the pin fails too
    assert abs(r0 - 1) >= 0.03 or abs(r2 - 1) >= 0.03 or abs(r2 / r0 - 1) >= 6e-3


def test_thermal_pin_catches_omega1():
    assert abs(thermal_mode(0.0, oracle_cls=mutation("omega1_is_omega").OracleLBM) - 1) >= 0.015


@pytest.mark.parametrize("name", ["qcorr_sign", "qcorr_factor", "qcorr_dropped",
                                  "qdiff_factor", "qdiff_half", "qdiff_dropped"])
def test_interdiffusion_pin_catches(name):
    try:
        drift = interdiffusion_T_drift(nx=32, nsteps=200,
                                       oracle_cls=mutation(name).OracleLBM)
    except thermo.NewtonError:
        return
    assert drift >= 5e-3


def test_r5_pin_catches_the_density_only_rule(monkeypatch):
    import oracle.boundary
    import oracle.lbm

    def density_only(rho_a, j_a):
        return rho_a <= oracle.lbm.RHO_TINY
    monkeypatch.setattr(oracle.lbm, "species_velocity_undefined", density_only)
    monkeypatch.setattr(oracle.boundary, "species_velocity_undefined", density_only)
    try:
        growth = _r5_growth()
    except thermo.NewtonError:
        return
    assert growth > 1.0e4
