"""Whole-step pins of the oracle (periodic boxes).

* Sec. 2.4 ("sub-iterations implement a zero-dimensional perfectly stirred
  reactor"): on a homogeneous box at rest, every node's species densities
  follow explicit Euler with step dt/l of the constant-volume, constant-
  energy reactor ODE exactly (to roundoff), written here as a plain loop.
* Sec. 3.8: in a closed periodic reactor total energy (incl. formation
  enthalpy) is constant and, without perturbation, no kinetic energy develops.
* Sec. 3.7: mass, momentum, each element and total energy are conserved on a
  periodic box with a perturbed state.
* Sec. 2.2 Eq. dtrhoa / Eq. constit2 (binary limit): two equal-mass inert
  species diffuse with the error-function profile of Fick's law at the
  model's D_12; the error falls at second order under refinement.
* Sec. 3.5 Eq. mu: a transverse shear wave decays at nu k^2 with
  nu = (1/omega - 1/2) theta.
* Sec. 2.3 Eq. transform1: the Householder QR solution solves the system.
"""
import numpy as np
import pytest

from lbm_workloads import fields
from lbm_workloads.mechanism import (P_STANDARD, R_UNIVERSAL, T_STANDARD,
                                     binary_inert, h2_air_synthetic)
from oracle import OracleLBM, thermo, chemistry


@pytest.fixture(scope="module")
def mech():
    return h2_air_synthetic()


def _make(mech, w, **kw):
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], T_max=w["T_max"],
                  substeps=w["substeps"], **kw)
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    return o, rho


def test_homogeneous_reactor_is_explicit_euler(mech):
    w = fields.reactor(n=2, T0=1400.0, perturbation=0.0, dx=2e-3)
    o, rho = _make(mech, w)
    nsteps, l = 25, w["substeps"]
    Y0 = w["Y"][:, 0, 0, 0]
    rho0 = rho[0, 0, 0]
    U = float(thermo.mixture_U(mech, Y0[:, None], np.array([1400.0]))[0])
    r = (rho0 * Y0)[:, None].copy()
    T = np.array([1400.0])
    dt = o.units.dt
    for _ in range(nsteps):
        T = thermo.temperature_from_energy(mech, r / rho0, np.array([U]), T)
        Ts = T
        for s in range(l):
            if s > 0:
                Ts = thermo.temperature_from_energy(mech, r / rho0, np.array([U]), Ts)
            r = r + dt / l * chemistry.production_rates(mech, Ts, r)
    o.step(nsteps)
    m = o.moments()
    got = m["rho"][0, 0, 0] * m["Y"][:, 0, 0, 0]
    assert np.max(np.abs(got - r[:, 0]) / np.maximum(np.abs(r[:, 0]), 1e-12)) < 1e-11
    assert np.all(np.abs(got - r[:, 0]) <= 1e-12 * rho0 + 1e-11 * np.abs(r[:, 0]))
    # the chemistry did something
    assert got[mech.index("H")] > 1e-9
    # closed reactor: no kinetic energy, total energy constant
    assert np.max(np.abs(m["u"])) < 1e-9
    E0 = U
    assert abs(m["E"][0, 0, 0] - E0) < 1e-12 * abs(E0) + 1e-6


def test_periodic_box_conserves_mass_momentum_elements_energy(mech):
    w = fields.reactor(n=4, T0=1400.0, perturbation=2e-2, seed=3, dx=1e-3)
    w["u"][0] = 3.0 * np.sin(2 * np.pi * np.arange(4) / 4)[None, None, :]
    o, _ = _make(mech, w)

    def totals():
        m = o.moments_of(o.pops)
        mass = m["rho"].sum()
        mom = m["j"].reshape(3, -1).sum(axis=1)
        energy = m["rhoE"].sum()
        moles = (m["rho_s"] / mech.molar_mass[:, None, None, None]).reshape(mech.n_species, -1)
        el = mech.composition.T @ moles.sum(axis=1)
        return mass, mom, energy, el
    m0, p0, e0, el0 = totals()
    o.step(12)
    m1, p1, e1, el1 = totals()
    assert abs(m1 - m0) <= 1e-14 * m0
    assert np.all(np.abs(p1 - p0) <= 1e-14 * m0)
    assert abs(e1 - e0) <= 1e-13 * abs(e0)
    assert np.all(np.abs(el1 - el0) <= 1e-13 * el0)
    # something moved and reacted
    assert np.max(np.abs(o.moments()["u"])) > 0.1


def _erf_profile(x, nx, Dt, lo=0.25, hi=0.75):
    from scipy.special import erf
    y = np.zeros_like(x, dtype=float)
    for k in (-1, 0, 1):
        x1, x2 = nx / 4 + k * nx, 3 * nx / 4 + k * nx
        y += 0.5 * (erf((x - x1) / (2 * np.sqrt(Dt))) - erf((x - x2) / (2 * np.sqrt(Dt))))
    return lo + (hi - lo) * y


def _binary_diffusion_error(W, lattice):
    mech = binary_inert()
    T0 = 300.0
    R = R_UNIVERSAL / mech.molar_mass[0]
    theta = 1.0 / 3.0
    c = np.sqrt(R * T0 / theta)
    # D_12 of the transport table at (T0, P0): power law in T (Sec. 3.6 stand-in)
    D = mech.D0[0, 1] * (T0 / T_STANDARD) ** mech.D_T_exponent
    D_lat_target = 0.05
    dx = D / (c * D_lat_target)
    D_lat = D * (dx / c) / dx ** 2
    nx = 16 * W
    o = OracleLBM(mech, lattice, (nx, 1, 1), dx, c_ref=c, substeps=1)
    x = np.arange(nx, dtype=float)
    Dt0 = (W / 2.0) ** 2
    t1 = int(round(1.25 * W * W / 4.0 / D_lat))
    YA = _erf_profile(x, nx, Dt0)
    Y = np.stack([YA, 1.0 - YA]).reshape(2, 1, 1, nx)
    rho = thermo.density_from_pressure(mech, P_STANDARD, T0, Y)
    o.init_fields(rho, np.zeros((3, 1, 1, nx)), np.full((1, 1, nx), T0), Y)
    o.step(t1)
    m = o.moments()
    ref = _erf_profile(x, nx, Dt0 + D_lat * t1)
    return np.max(np.abs(m["Y"][0, 0, 0] - ref)) / 0.5, np.max(np.abs(m["u"]))


@pytest.mark.slow
@pytest.mark.parametrize("lattice", ["D3Q27", "D2Q9"])
def test_binary_diffusion_erf_profile(lattice):
    e4, u4 = _binary_diffusion_error(4, lattice)
    e8, u8 = _binary_diffusion_error(8, lattice)
    assert e8 < 1.0e-3
    assert e4 / e8 > 3.0                     # second order: ratio 4
    assert max(u4, u8) < 1e-9                # equal masses: no mixture flow


@pytest.mark.slow
def test_shear_wave_viscosity():
    mech = binary_inert()
    T = 300.0
    R = R_UNIVERSAL / mech.molar_mass[0]
    c = np.sqrt(R * T / 0.3)
    w = fields.shear_wave(nx=48, amplitude=0.5, T=T, dx=2e-7, mech=mech)
    o = OracleLBM(mech, "D3Q27", w["shape"], w["dx"], c_ref=c, substeps=1)
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    from oracle.transport import relaxation
    rel = relaxation(mech, o.units, rho, w["Y"], w["T"])
    omega, theta = rel["omega"].ravel()[0], rel["theta"].ravel()[0]
    nu = (1.0 / omega - 0.5) * theta
    k = 2 * np.pi / 48
    amp = []
    for _ in range(3):
        o.step(40)
        uy = o.moments()["u"][1, 0, 0] / o.units.c
        amp.append(2.0 / 48 * np.sum(uy * np.sin(k * np.arange(48))))
    rate = np.log(amp[1] / amp[2]) / 40.0
    assert abs(rate / (nu * k * k) - 1.0) < 0.01


def test_householder_solution_solves_system(mech):
    w = fields.reactor(n=2, T0=1300.0, perturbation=0.0)
    o, rho = _make(mech, w)
    rng = np.random.default_rng(5)
    M = mech.n_species
    Y = rng.dirichlet(np.ones(M), size=8).T.reshape(M, 2, 2, 2)
    inv_tau_ab = rng.uniform(0.1, 3.0, size=(M, M, 2, 2, 2))
    inv_tau_ab = 0.5 * (inv_tau_ab + inv_tau_ab.transpose(1, 0, 2, 3, 4))
    for a in range(M):
        inv_tau_ab[a, a] = 0.0
    inv_tau_a = np.einsum("b...,ab...->a...", Y, inv_tau_ab)
    rhs = rng.normal(size=(M, 3, 2, 2, 2))
    V = o.diffusion_velocities(Y, inv_tau_ab, inv_tau_a, rhs)
    for n in np.ndindex(2, 2, 2):
        A = np.diag(1.0 + 0.5 * inv_tau_a[(slice(None),) + n])
        for a in range(M):
            for b in range(M):
                if a != b:
                    A[a, b] = -0.5 * Y[(b,) + n] * inv_tau_ab[(a, b) + n]
        for al in range(3):
            x = V[(slice(None), al) + n]
            assert np.allclose(A @ x, rhs[(slice(None), al) + n], atol=1e-14)
            assert np.allclose(x, np.linalg.solve(A, rhs[(slice(None), al) + n]), atol=1e-13)
