"""Reaction rates of the mechanism table and the per-node reactor sub-steps.

Test infrastructure: plain FP64 numpy.

* Rates (what Cantera supplies in Sec. 3.6): for reaction r,
  k_f = A T^b exp(-Ea/(R_U T)); concentrations C_a = rho_a/m_a;
  a third body contributes [M] = sum_a eff_ra C_a;
  reverse rate k_r = k_f / K_c with
  K_c = exp(-sum_a nu_a g_a(T)/(R_U T)) (P0/(R_U T))^(sum_a nu_a),
  nu = nu_r - nu_f, g_a = h_a - T s_a of the table's thermodynamics;
  q_r = [M] (k_f prod C^nu_f - k_r prod C^nu_r);
  rho_dot_a = m_a sum_r nu_ra q_r  (kg/(m^3 s)).  Mass conservation,
  Eq. sumRhoDot, holds because every reaction is element balanced.
* Sub-steps, Sec. 2.4 Eq. R3: with the internal energy U frozen,
  l forward-Euler steps of length dt/l:
  T_s = T(U, Y^(s)), rho^(s+1) = rho^(s) + (dt/l) rho_dot(T_s, rho^(s)).
"""
import numpy as np

from lbm_workloads.mechanism import R_UNIVERSAL, P_STANDARD
from . import thermo


def forward_rate_constants(mech, T):
    """k_f per reaction, shape [R, ...] (the Arrhenius form that stands in
    for Cantera's rates, Sec. 3.6; readings R17)."""
    T = np.asarray(T, dtype=float)
    A = mech.arrhenius[:, 0].reshape((-1,) + (1,) * T.ndim)
    b = mech.arrhenius[:, 1].reshape((-1,) + (1,) * T.ndim)
    Ea = mech.arrhenius[:, 2].reshape((-1,) + (1,) * T.ndim)
    return A * T ** b * np.exp(-Ea / (R_UNIVERSAL * T))


def equilibrium_constants(mech, T):
    """K_c per reaction (concentration units), shape [R, ...]: the table's own
    equilibrium constants, which make the reverse rates consistent with the
    thermodynamics of Sec. 3.1."""
    T = np.asarray(T, dtype=float)
    g = thermo.h_molar(mech, T) - T * thermo.s_molar(mech, T)      # [M, ...]
    nu = mech.nu_r - mech.nu_f                                      # [R, M]
    dG = np.tensordot(nu, g, axes=(1, 0))                           # [R, ...]
    dn = nu.sum(axis=1).reshape((-1,) + (1,) * T.ndim)
    return np.exp(-dG / (R_UNIVERSAL * T)) * (P_STANDARD / (R_UNIVERSAL * T)) ** dn


def rates_of_progress(mech, T, rho_species):
    """q_r (mol/(m^3 s)), shape [R, ...] (rates of progress for Sec. 2.4; third
    bodies and reverse rates as in the module docstring).  rho_species: [M, ...] (kg/m^3)."""
    T = np.asarray(T, dtype=float)
    shape = T.shape
    C = rho_species / mech.molar_mass.reshape((-1,) + (1,) * T.ndim)  # [M, ...]
    kf = forward_rate_constants(mech, T)
    Kc = equilibrium_constants(mech, T)
    q = np.zeros((mech.n_reactions,) + shape)
    for r in range(mech.n_reactions):
        fwd = kf[r] * np.ones(shape)
        for a in range(mech.n_species):
            for _ in range(int(mech.nu_f[r, a])):
                fwd = fwd * C[a]
        rev = np.zeros(shape)
        if mech.reversible[r]:
            rev = kf[r] / Kc[r] * np.ones(shape)
            for a in range(mech.n_species):
                for _ in range(int(mech.nu_r[r, a])):
                    rev = rev * C[a]
        qr = fwd - rev
        if mech.third_body[r]:
            conc_M = np.tensordot(mech.efficiency[r], C, axes=(0, 0))
            qr = qr * conc_M
        q[r] = qr
    return q


def production_rates(mech, T, rho_species):
    """rho_dot_a (kg/(m^3 s)), shape [M, ...]: the mass production rates of
    Sec. 2.4 (their sum vanishes, Eq. sumRhoDot)."""
    q = rates_of_progress(mech, T, rho_species)
    nu = mech.nu_r - mech.nu_f                                       # [R, M]
    wdot = np.tensordot(nu, q, axes=(0, 0))                          # [M, ...]
    return wdot * mech.molar_mass.reshape((-1,) + (1,) * np.ndim(T))


def reactor_substeps(mech, rho_species, U, T_start, dt, l, rtol=1e-13, max_iter=50):
    """Eq. R3: l forward-Euler sub-steps at frozen internal energy U.

    rho_species: [M, ...] kg/m^3; U: [...] J/kg (sensible + formation);
    T_start: temperature of the initial composition (used as T_0 and as the
    Newton start of later sub-steps); dt: fluid time step (s).
    Returns (delta_rho [M, ...], list of the sub-step temperatures).
    """
    rho = np.sum(rho_species, axis=0)
    r = np.array(rho_species, dtype=float, copy=True)
    dtr = dt / l
    T = np.array(T_start, dtype=float, copy=True)
    temps = []
    for s in range(l):
        if s > 0:
            T = thermo.temperature_from_energy(mech, r / rho, U, T, rtol, max_iter)
        temps.append(T)
        r = r + dtr * production_rates(mech, T, r)
    return r - rho_species, temps
