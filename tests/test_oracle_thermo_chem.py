"""Pins of the oracle's thermodynamics, temperature solve and reaction rates.

* Sec. 3.1: dH_a/dT = C_ap and dU_a/dT = C_av (finite differences of the
  energies, not the heat-capacity formulas), C_ap - C_av = R_a, H_a(T0) =
  formation enthalpy; constant-c_p species have the closed-form inverse
  T = T0 + (U - U^0)/C_v.
* Eq. temperature: Newton round trip T -> U(T) -> T from a distant start.
* Eq. sumRhoDot: reactions conserve mass; each reaction of the table
  balances every element.
* Chemical equilibrium of the table: integrating the constant-volume reactor
  to steady state drives every reaction's affinity sum_a nu_a mu_a to zero,
  with mu_a = g_a(T) + R_U T ln(C_a R_U T / P0) from the textbook definition
  (this checks the equilibrium constants' sign and exponent conventions).
* Eq. R3 sub-steps against a tight-tolerance stiff ODE integration of the
  same reactor: first-order convergence in dt/l.
"""
import numpy as np
import pytest

from lbm_workloads.mechanism import (R_UNIVERSAL, T_STANDARD, P_STANDARD,
                                     h2_air_synthetic, binary_inert,
                                     air_mole_fractions, mole_to_mass_fractions)
from oracle import thermo, chemistry


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def test_energy_derivatives_are_heat_capacities(mech):
    T = np.array([300.0, 900.0, 1700.0, 2900.0])
    h = 1e-3
    dH = (thermo.H_species(mech, T + h) - thermo.H_species(mech, T - h)) / (2 * h)
    dU = (thermo.U_species(mech, T + h) - thermo.U_species(mech, T - h)) / (2 * h)
    cp_mass = thermo.cp_molar(mech, T) / mech.molar_mass[:, None]
    assert np.allclose(dH, cp_mass, rtol=1e-7)
    assert np.allclose(dU, thermo.Cv_species(mech, T), rtol=1e-7)
    assert np.allclose(cp_mass - thermo.Cv_species(mech, T),
                       (R_UNIVERSAL / mech.molar_mass)[:, None], rtol=1e-13)
    H0 = thermo.H_species(mech, np.array([T_STANDARD]))[:, 0]
    assert np.allclose(H0, mech.h_formation / mech.molar_mass, atol=1e-9)
    ds = (thermo.s_molar(mech, T + h) - thermo.s_molar(mech, T - h)) / (2 * h)
    assert np.allclose(ds, thermo.cp_molar(mech, T) / T, rtol=1e-7)


def test_temperature_newton_round_trip(mech):
    rng = np.random.default_rng(3)
    Y = rng.dirichlet(np.ones(mech.n_species), size=50).T          # [M, 50]
    T = rng.uniform(250.0, 3200.0, 50)
    U = thermo.mixture_U(mech, Y, T)
    T_back = thermo.temperature_from_energy(mech, Y, U, np.full(50, 1000.0))
    assert np.max(np.abs(T_back - T) / T) < 1e-13


def test_temperature_constant_cp_closed_form():
    mech = binary_inert(cp_over_R=3.5)
    Y = np.array([[0.3], [0.7]])
    U = np.array([2.0e5])
    cv = (3.5 - 1.0) * R_UNIVERSAL / mech.molar_mass[0]
    U0 = -R_UNIVERSAL / mech.molar_mass[0] * T_STANDARD        # h_f = 0
    T = thermo.temperature_from_energy(mech, Y, U, np.array([500.0]))
    assert abs(T[0] - (T_STANDARD + (U[0] - U0) / cv)) < 1e-10


def test_newton_failure_raises(mech):
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, 0.5))[:, None]
    with pytest.raises(thermo.NewtonError):
        thermo.temperature_from_energy(mech, Y, np.array([1e6]), np.array([300.0]),
                                       max_iter=0 + 1, rtol=0.0)


def test_reactions_balance_elements_and_mass(mech):
    nu = mech.nu_r - mech.nu_f
    assert mech.n_reactions == 21 and mech.n_species == 9
    assert np.all(nu @ mech.composition == 0)
    assert np.max(np.abs(nu @ mech.molar_mass)) < 1e-15 * mech.molar_mass.max()
    rng = np.random.default_rng(4)
    rho_s = rng.uniform(0.0, 0.05, size=(9, 40))
    T = rng.uniform(800.0, 2500.0, 40)
    wdot = chemistry.production_rates(mech, T, rho_s)
    scale = np.max(np.abs(wdot), axis=0)
    assert np.all(np.abs(wdot.sum(axis=0)) <= 1e-12 * scale)


def _reactor_rhs(mech, rho, U):
    def rhs(t, r):
        T = thermo.temperature_from_energy(mech, (r / rho)[:, None], np.array([U]),
                                           np.array([rhs.T]))
        rhs.T = T[0]
        return chemistry.production_rates(mech, T, r[:, None])[:, 0]
    rhs.T = 1200.0
    return rhs


def _initial_state(mech, phi=0.5, T=1200.0):
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, phi))
    rho = thermo.density_from_pressure(mech, P_STANDARD, T, Y)
    U = float(thermo.mixture_U(mech, Y[:, None], np.array([T]))[0])
    return rho, rho * Y, U


@pytest.mark.slow
def test_chemical_equilibrium_affinities_vanish(mech):
    scipy = pytest.importorskip("scipy.integrate")
    rho, r0, U = _initial_state(mech, phi=0.5, T=1400.0)
    rhs = _reactor_rhs(mech, rho, U)
    sol = scipy.solve_ivp(rhs, (0.0, 1.0), r0, method="Radau", rtol=1e-10,
                          atol=1e-16)
    r = sol.y[:, -1]
    T = thermo.temperature_from_energy(mech, (r / rho)[:, None], np.array([U]),
                                       np.array([2000.0]))[0]
    # element totals unchanged
    n0 = (r0 / mech.molar_mass) @ mech.composition
    n1 = (r / mech.molar_mass) @ mech.composition
    assert np.allclose(n0, n1, rtol=1e-8)
    assert T > 1400.0 + 300.0                    # the lean mixture has burnt
    C = r / mech.molar_mass
    g = thermo.h_molar(mech, np.array([T]))[:, 0] - T * thermo.s_molar(mech, np.array([T]))[:, 0]
    mu = g + R_UNIVERSAL * T * np.log(C * R_UNIVERSAL * T / P_STANDARD)
    nu = mech.nu_r - mech.nu_f
    affinity = nu @ mu                             # J/mol
    assert np.max(np.abs(affinity)) < 1e-3 * R_UNIVERSAL * T
    q = chemistry.rates_of_progress(mech, np.array([T]), r[:, None])[:, 0]
    kf = chemistry.forward_rate_constants(mech, np.array([T]))[:, 0]
    fwd = np.array([kf[k] * np.prod(C ** mech.nu_f[k]) for k in range(mech.n_reactions)])
    fwd = fwd * np.where(mech.third_body == 1, mech.efficiency @ C, 1.0)
    assert np.all(np.abs(q) <= 1e-3 * fwd)


@pytest.mark.slow
def test_substeps_converge_to_stiff_reactor_solution(mech):
    """Explicit sub-steps (Eq. R3) converge at first order in dt/l to the
    tight-tolerance Radau solution of the same constant-U reactor."""
    scipy = pytest.importorskip("scipy.integrate")
    rho, r0, U = _initial_state(mech, phi=0.5, T=1300.0)
    t_end = 2.0e-5
    rhs = _reactor_rhs(mech, rho, U)
    ref = scipy.solve_ivp(rhs, (0.0, t_end), r0, method="Radau", rtol=1e-12,
                          atol=1e-18).y[:, -1]
    iOH = mech.index("OH")
    errs = []
    for n in (200, 400, 800):
        r = r0[:, None].copy()
        T = np.array([1300.0])
        dt = t_end / n
        for _ in range(n):
            dr, temps = chemistry.reactor_substeps(mech, r, np.array([U]), T, dt, 1)
            r = r + dr
            T = thermo.temperature_from_energy(mech, r / rho, np.array([U]), T)
        errs.append(abs(r[iOH, 0] - ref[iOH]) / abs(ref[iOH]))
    order1 = np.log2(errs[0] / errs[1])
    order2 = np.log2(errs[1] / errs[2])
    assert 0.8 < order1 < 1.3 and 0.8 < order2 < 1.3, errs


# --- Wilke mixing rule (the transport option of the viscosity model) -------

def test_wilke_single_species_is_its_own_viscosity():
    """Phi_aa = 1, so a pure species has its own viscosity at any T."""
    from lbm_workloads.mechanism import h2_air_synthetic, with_viscosity_model
    from oracle import transport
    m = with_viscosity_model(h2_air_synthetic(), "wilke")
    for a in range(m.n_species):
        Y = np.zeros((m.n_species, 1))
        Y[a] = 1.0
        mu = transport.viscosity(m, np.array([900.0]), Y)[0]
        want = m.mu0_species[a] * (900.0 / 298.15) ** m.mu_T_exponent
        assert mu == pytest.approx(want, rel=1e-14)


def test_wilke_binary_mixture_textbook_form():
    """Two species: mu = X1 mu1/(X1 + X2 Phi12) + X2 mu2/(X1 Phi21 + X2),
    with Phi21 = Phi12 (mu2/mu1)(m1/m2) (the symmetry of Wilke's Phi)."""
    from lbm_workloads.mechanism import h2_air_synthetic, with_viscosity_model
    from oracle import transport
    m = with_viscosity_model(h2_air_synthetic(), "wilke")
    i, j = m.species.index("H2"), m.species.index("N2")
    Y = np.zeros((m.n_species, 1))
    Y[i], Y[j] = 0.03, 0.97
    mu = transport.viscosity(m, np.array([298.15]), Y)[0]
    m1, m2 = m.molar_mass[i], m.molar_mass[j]
    u1, u2 = m.mu0_species[i], m.mu0_species[j]
    x1 = (0.03 / m1) / (0.03 / m1 + 0.97 / m2)
    x2 = 1.0 - x1
    phi12 = (1 + np.sqrt(u1 / u2) * (m2 / m1) ** 0.25) ** 2 / np.sqrt(8 * (1 + m1 / m2))
    phi21 = phi12 * (u2 / u1) * (m1 / m2)
    want = x1 * u1 / (x1 + x2 * phi12) + x2 * u2 / (x1 * phi21 + x2)
    assert mu == pytest.approx(want, rel=1e-13)
    assert min(u1, u2) < mu < max(u1, u2)


def test_wilke_equal_species_recover_the_mixture_model():
    """Species of equal mass and viscosity: Phi = 1 everywhere, mu = mu_a."""
    from lbm_workloads.mechanism import binary_inert, with_viscosity_model
    from oracle import transport
    m = with_viscosity_model(binary_inert(), "wilke")
    Y = np.array([[0.3], [0.7]])
    mu_w = transport.viscosity(m, np.array([700.0]), Y)[0]
    mu_m = transport.viscosity(binary_inert(), np.array([700.0]))[0]
    assert mu_w == pytest.approx(mu_m, rel=1e-15)
