"""Transport model and the relaxation parameters of the lattice equations.

Test infrastructure: plain FP64 numpy.

The paper takes mu, lambda and D_ab from Cantera (Sec. 3.5 end, Sec. 3.6).
Cantera is not available, so the mechanism table carries a power-law model:
D_ab = D0_ab (T/T0)^{D_T_exponent} (P0/P), mu = mu0 (T/T0)^{mu_T_exponent}
(or, as an option, Wilke's mixing rule over species viscosities),
lambda = mu C_p / Pr.

Relaxation parameters in lattice units (dx = dt = 1, velocities scaled by
the reference speed c, theta_a = R_a T / c^2, theta = R T / c^2):

* Sec. 2.3, Eqs. betaa and taua, with the characteristic time read as
  tau_ab = D_ab m_a m_b / (m R_U T) (the printed ratio is its inverse, a
  rate; only this form makes 1/tau_a = sum Y_b/tau_ab equal the kinetic
  relaxation rate sum_b P X_a X_b/(D_ab rho_a) of Eq. stefanMaxwell).
  In lattice units tau_ab = D_lat m_b / (m theta_a), D_lat = D dt/dx^2.
  1/tau_a = sum_{b != a} Y_b / tau_ab, beta_a = 1/(2 tau_a + 1).
* Sec. 3.5, Eq. mu: mu = (1/omega - 1/2) P dt  =>  1/omega = nu_lat/theta + 1/2.
* Sec. 3.5, Eq. lambda: lambda = (1/omega1 - 1/2) P C_p dt
  =>  1/omega1 = alpha_lat/theta + 1/2 with alpha = lambda/(rho C_p) = nu/Pr.
"""
import numpy as np

from lbm_workloads.mechanism import R_UNIVERSAL, T_STANDARD, P_STANDARD


def diffusion_coefficients(mech, T, P):
    """D_ab (m^2/s), shape [M, M, ...] (the power law of reading R9, standing in
    for Cantera's binary coefficients, Sec. 3.6)."""
    T = np.asarray(T, dtype=float)
    s = (T / T_STANDARD) ** mech.D_T_exponent * (P_STANDARD / P)
    return mech.D0.reshape(mech.D0.shape + (1,) * T.ndim) * s


def viscosity(mech, T, Y=None):
    """Mixture viscosity (Pa s), reading R9 (Sec. 3.5 takes it from Cantera).  "mixture" model: mu0 (T/T0)^e.  "wilke"
    model (Wilke's mixing rule, J. Chem. Phys. 18, 1950) over the species
    viscosities mu_a = mu0_a (T/T0)^e:
      mu = sum_a X_a mu_a / sum_b X_b Phi_ab,
      Phi_ab = [1 + (mu_a/mu_b)^(1/2) (m_b/m_a)^(1/4)]^2 / [8 (1 + m_a/m_b)]^(1/2),
    with X the mole fractions of Y [M, ...]."""
    T = np.asarray(T, dtype=float)
    scale = (T / T_STANDARD) ** mech.mu_T_exponent
    if mech.viscosity_model != "wilke":
        return mech.mu0 * scale
    M = mech.n_species
    m = mech.molar_mass
    Y = np.asarray(Y, dtype=float)
    n = Y / m.reshape((-1,) + (1,) * (Y.ndim - 1))
    X = n / np.sum(n, axis=0)
    mu_a = [mech.mu0_species[a] * scale for a in range(M)]
    total = np.zeros(T.shape)
    for a in range(M):
        den = np.zeros(T.shape)
        for b in range(M):
            phi = (1.0 + np.sqrt(mu_a[a] / mu_a[b]) * (m[b] / m[a]) ** 0.25) ** 2 \
                / np.sqrt(8.0 * (1.0 + m[a] / m[b]))
            den = den + X[b] * phi
        total = total + X[a] * mu_a[a] / den
    return total


def relaxation(mech, units, rho, Y, T):
    """Per-node relaxation data (Sec. 2.3 Eqs. betaa, taua; Sec. 3.5 Eqs. mu,
    lambda; reading R3).

    Returns dict with inv_tau_ab [M, M, ...] (zero diagonal), inv_tau_a [M, ...],
    beta [M, ...], omega [...], omega1 [...].
    """
    from . import thermo
    T = np.asarray(T, dtype=float)
    R = thermo.mixture_gas_constant(mech, Y)
    P = rho * R * T                                          # Pa
    m = R_UNIVERSAL / R                                      # mixture molar mass
    c2 = units.c ** 2
    Ra = thermo.species_gas_constant(mech)
    theta_a = Ra.reshape((-1,) + (1,) * T.ndim) * T / c2     # [M, ...]
    D = diffusion_coefficients(mech, T, P)                   # [M, M, ...]
    D_lat = D * units.dt / units.dx ** 2
    M = mech.n_species
    inv_tau_ab = np.zeros((M, M) + T.shape)
    for a in range(M):
        for b in range(M):
            if a != b:
                tau_ab = D_lat[a, b] * mech.molar_mass[b] / (m * theta_a[a])
                inv_tau_ab[a, b] = 1.0 / tau_ab
    inv_tau_a = np.zeros((M,) + T.shape)
    for a in range(M):
        for b in range(M):
            if b != a:
                inv_tau_a[a] = inv_tau_a[a] + Y[b] * inv_tau_ab[a, b]
    beta = inv_tau_a / (2.0 + inv_tau_a)                     # = 1/(2 tau_a + 1)
    theta = R * T / c2
    nu_lat = viscosity(mech, T, Y) / rho * units.dt / units.dx ** 2
    omega = 1.0 / (nu_lat / theta + 0.5)
    omega1 = 1.0 / (nu_lat / (mech.prandtl * theta) + 0.5)
    return dict(inv_tau_ab=inv_tau_ab, inv_tau_a=inv_tau_a, beta=beta,
                omega=omega, omega1=omega1, theta_a=theta_a, theta=theta, P=P)
