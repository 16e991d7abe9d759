"""Thermodynamics of the ideal-gas mixture and the temperature solve.

Test infrastructure: plain FP64 numpy.

* Mixture relations of Sec. 2.1: rho = sum rho_a, Y_a = rho_a/rho,
  1/m = sum Y_a/m_a, P = rho R T with R = R_U/m, R_a = R_U/m_a.
* Species energies of Sec. 3.1 (Eqs. specUa, specHa, U, H):
  U_a = U_a^0 + int_T0^T C_av dT', H_a = H_a^0 + int_T0^T C_ap dT',
  C_ap - C_av = R_a.  With the formation enthalpy h_f at T0 per mole,
  H_a(T) = (h_f + R_U int_T0^T c_p/R_U dT') / m_a and U_a = H_a - R_a T
  (so U_a^0 = H_a^0 - R_a T0).
* Temperature from energy, Eq. temperature: solve sum_a Y_a U_a(T) = U by
  Newton's method, F'(T) = sum_a Y_a C_av(T); warm start from the previous T,
  stop when |dT| <= rtol*T (reading R11: rtol = 1e-13, at most 50 iterations).
"""
import numpy as np

from lbm_workloads.mechanism import R_UNIVERSAL, T_STANDARD, P_STANDARD


class NewtonError(RuntimeError):
    """The temperature Newton of Eq. temperature did not converge (reading R11)."""


def cp_molar(mech, T):
    """c_p (J/(mol K)) per species, shape [M, ...] (Sec. 3.1, the table's
    polynomial, reading R17)."""
    T = np.asarray(T, dtype=float)
    a = mech.cp_coeffs
    return R_UNIVERSAL * (a[:, 0, None] + a[:, 1, None] * T.ravel()[None]
                          + a[:, 2, None] * T.ravel()[None] ** 2).reshape((-1,) + T.shape)


def h_molar(mech, T):
    """Molar enthalpy incl. formation, h = h_f + int_T0^T c_p dT' (J/mol)
    (Sec. 3.1, Eq. specHa per mole)."""
    T = np.asarray(T, dtype=float)
    a = mech.cp_coeffs
    t, t0 = T.ravel()[None], T_STANDARD
    integral = (a[:, 0, None] * (t - t0) + a[:, 1, None] / 2.0 * (t ** 2 - t0 ** 2)
                + a[:, 2, None] / 3.0 * (t ** 3 - t0 ** 3))
    return (mech.h_formation[:, None] + R_UNIVERSAL * integral).reshape((-1,) + T.shape)


def s_molar(mech, T):
    """Standard-state molar entropy s = s0 + int_T0^T c_p/T' dT' (J/(mol K));
    enters the equilibrium constants of the reverse rates (Sec. 2.4)."""
    T = np.asarray(T, dtype=float)
    a = mech.cp_coeffs
    t, t0 = T.ravel()[None], T_STANDARD
    integral = (a[:, 0, None] * np.log(t / t0) + a[:, 1, None] * (t - t0)
                + a[:, 2, None] / 2.0 * (t ** 2 - t0 ** 2))
    return (mech.s_standard[:, None] + R_UNIVERSAL * integral).reshape((-1,) + T.shape)


def species_gas_constant(mech):
    """R_a = R_U / m_a (Sec. 2.1)."""
    return R_UNIVERSAL / mech.molar_mass                       # R_a, J/(kg K)


def H_species(mech, T):
    """Mass-specific enthalpy H_a (J/kg), shape [M, ...] (Sec. 3.1, Eq. specHa)."""
    mm = mech.molar_mass.reshape((-1,) + (1,) * np.ndim(T))
    return h_molar(mech, T) / mm


def U_species(mech, T):
    """Mass-specific internal energy U_a = H_a - R_a T (J/kg) (Sec. 3.1,
    Eq. specUa)."""
    Ra = species_gas_constant(mech).reshape((-1,) + (1,) * np.ndim(T))
    return H_species(mech, T) - Ra * np.asarray(T)


def Cv_species(mech, T):
    """Mass-specific C_av = C_ap - R_a (Mayer relation), J/(kg K) (Sec. 3.1)."""
    mm = mech.molar_mass.reshape((-1,) + (1,) * np.ndim(T))
    Ra = species_gas_constant(mech).reshape((-1,) + (1,) * np.ndim(T))
    return cp_molar(mech, T) / mm - Ra


def mixture_gas_constant(mech, Y):
    """R = R_U / m with 1/m = sum_a Y_a/m_a (Sec. 2.1).  Y: [M, ...]."""
    mm = mech.molar_mass.reshape((-1,) + (1,) * (np.ndim(Y) - 1))
    return R_UNIVERSAL * np.sum(Y / mm, axis=0)


def mixture_U(mech, Y, T):
    """U = sum_a Y_a U_a (Sec. 3.1, Eq. U)."""
    return np.sum(Y * U_species(mech, T), axis=0)


def mixture_H(mech, Y, T):
    """H = sum_a Y_a H_a (Sec. 3.1, Eq. H)."""
    return np.sum(Y * H_species(mech, T), axis=0)


def mixture_Cv(mech, Y, T):
    """C_v = sum_a Y_a C_av (Sec. 3.1), the Newton derivative of Eq. temperature."""
    return np.sum(Y * Cv_species(mech, T), axis=0)


def density_from_pressure(mech, P, T, Y):
    """rho = P / (R T)  (Eq. eosIdealGas)."""
    return P / (mixture_gas_constant(mech, Y) * T)


def temperature_from_energy(mech, Y, U, T_guess, rtol=1e-13, max_iter=50):
    """Solve sum_a Y_a U_a(T) = U for T by Newton (Eq. temperature).

    Y: [M, ...], U and T_guess: [...] (J/kg, K).  Every node iterates until
    its own |dT| <= rtol*T; a node that has not converged after max_iter
    iterations raises NewtonError.
    """
    T = np.array(T_guess, dtype=float, copy=True)
    U = np.asarray(U, dtype=float)
    active = np.ones(T.shape, dtype=bool)
    for _ in range(max_iter):
        if not active.any():
            return T
        F = mixture_U(mech, Y, T) - U
        dF = mixture_Cv(mech, Y, T)
        dT = -F / dF
        T = np.where(active, T + dT, T)
        active = active & ~(np.abs(dT) <= rtol * np.abs(T))
    if active.any():
        raise NewtonError(f"temperature Newton did not converge at {int(active.sum())} nodes")
    return T


__all__ = ["cp_molar", "h_molar", "s_molar", "species_gas_constant", "H_species",
           "U_species", "Cv_species", "mixture_gas_constant", "mixture_U",
           "mixture_H", "mixture_Cv", "density_from_pressure",
           "temperature_from_energy", "NewtonError", "P_STANDARD"]
