"""Pins of the oracle's flame diagnostics (Sec. 5.3 quantities) against what
the thermodynamics and the definitions fix."""
import numpy as np
import pytest

from lbm_workloads.mechanism import h2_air_synthetic, air_mole_fractions, mole_to_mass_fractions
from oracle import chemistry, diagnostics, thermo


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _radical_state(mech, T=1500.0, rho=0.3):
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, 0.5))
    i = {s: k for k, s in enumerate(mech.species)}
    Y = Y.copy()
    for s, y in (("H", 1e-4), ("O", 2e-4), ("OH", 1e-3), ("HO2", 1e-5), ("H2O", 0.05)):
        Y[i[s]] = y
    Y[i["N2"]] += 1.0 - Y.sum()
    return T, rho, Y


def test_heat_release_matches_the_temperature_rise_of_a_closed_reactor(mech):
    """In a closed adiabatic constant-volume reactor U is fixed, so
    rho c_v dT/dt = -sum_a U_a rho_dot_a; with H_a = U_a + R_a T the enthalpy
    form is q = rho c_v dT/dt - T sum_a R_a rho_dot_a.  The temperature rise
    comes from the Newton solve of Eq. temperature at the new composition, a
    routine independent of the enthalpy sum."""
    T, rho, Y = _radical_state(mech)
    rs = rho * Y
    q = diagnostics.heat_release_rate(mech, np.array([T]), rs[:, None])[0]
    wdot = chemistry.production_rates(mech, np.array([T]), rs[:, None])[:, 0]
    dt = 1e-9
    U = thermo.mixture_U(mech, Y, T)
    Y2 = (rs + dt * wdot) / rho
    T2 = thermo.temperature_from_energy(mech, Y2, U, T)
    cv = thermo.mixture_Cv(mech, Y, T)
    Ra = thermo.species_gas_constant(mech)
    expected = rho * cv * (T2 - T) / dt - T * np.sum(Ra * wdot)
    assert abs(q) > 1e3
    assert q == pytest.approx(expected, rel=2e-5)


def test_no_heat_release_without_reaction(mech):
    """Pure N2 (inert in every reaction as a product or reactant): no rates."""
    Y = np.zeros(mech.n_species)
    Y[mech.species.index("N2")] = 1.0
    q = diagnostics.heat_release_rate(mech, np.array([1800.0]), (0.2 * Y)[:, None])
    assert q[0] == 0.0


def test_integral_position_and_maxima_on_a_constructed_field(mech):
    """A 6x2x2 field, reacting only at x = 3 (both planes identical): the
    integral is the sum times dx^3, the flame sits at 3 dx, the maxima are the
    field's."""
    nx, ny, nz, dx = 6, 2, 2, 1e-4
    N = nx * ny * nz
    T0, rho0, Yr = _radical_state(mech)
    Yc = np.zeros(mech.n_species)
    Yc[mech.species.index("N2")] = 1.0
    Y = np.repeat(Yc[:, None], N, axis=1)
    T = np.full(N, 600.0)
    rho = np.full(N, rho0)
    x = np.arange(N) % nx
    Y[:, x == 3] = Yr[:, None]
    T[x == 3] = T0
    u = np.zeros((3, N))
    u[0, 5] = -2.0
    u[1, 5] = 1.5
    d = diagnostics.diagnostics(mech, rho, u, T, Y, dx, 3, nx)
    q_node = diagnostics.heat_release_rate(mech, np.array([T0]), (rho0 * Yr)[:, None])[0]
    assert d["hrr_integral"] == pytest.approx(4 * q_node * dx ** 3, rel=1e-14)
    assert d["hrr_max"] == pytest.approx(q_node, rel=1e-15)
    assert d["flame_x"] == pytest.approx(3 * dx)
    assert d["T_max"] == T0
    assert d["u_max"] == pytest.approx(2.5)
