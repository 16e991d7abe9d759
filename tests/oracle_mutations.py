"""Planted mistakes in the oracle, on the CPU, for the pins' own tests.

A pin is worth its name only if a plausible mistake in the oracle makes it
fail.  ``mutated_oracle`` loads a copy of an oracle module with one exact
piece of its source replaced (a flipped sign, a wrong factor, a dropped
term) and returns the copy; the oracle package itself is never modified.
"""
import os
import types

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                          "oracle")


def mutated_oracle(old, new, module="lbm"):
    """A copy of oracle/<module>.py with the single occurrence of `old`
    replaced by `new`; relative imports resolve inside the oracle package."""
    path = os.path.join(ORACLE_DIR, module + ".py")
    src = open(path).read()
    n = src.count(old)
    if n != 1:
        raise ValueError(f"{old!r} occurs {n} times in {path}")
    mod = types.ModuleType(f"oracle._mutated_{module}")
    mod.__package__ = "oracle"
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    return mod


# Mistakes in the momentum and energy lattices' collision (oracle/lbm.py):
# (name, source text, replacement).
MUTATIONS = {
    # Eq. Pex: the extension's factor (2 - omega)/(2 rho omega)
    "Pex_dropped": ("(2.0 - omega) / (2.0 * rho * omega) * dPhi[a]", "0.0 * dPhi[a]"),
    "Pex_half": ("(2.0 - omega) / (2.0 * rho * omega) * dPhi[a]",
                 "0.5 * (2.0 - omega) / (2.0 * rho * omega) * dPhi[a]"),
    # Eq. qex: the energy flux of the extension
    "qex_sign": ("q_ex = np.array([-0.5 * u[a] * dPhi[a]", "q_ex = np.array([0.5 * u[a] * dPhi[a]"),
    "qex_dropped": ("q_ex = np.array([-0.5 * u[a] * dPhi[a]",
                    "q_ex = np.array([0.0 * u[a] * dPhi[a]"),
    # Eq. gstareq1mom: the u.(P - P^eq) term of q^*
    "uP_sign": ('mom["q"] - q_eq - uP + q_ex', 'mom["q"] - q_eq + uP + q_ex'),
    "uP_dropped": ('mom["q"] - q_eq - uP + q_ex', 'mom["q"] - q_eq + q_ex'),
    # Eq. lambda: omega_1 from the conductivity (here replaced by omega, Pr = 1)
    "omega1_is_omega": ('omega, omega1 = rel["omega"], rel["omega1"]',
                        'omega, omega1 = rel["omega"], rel["omega"]'),
    # Eq. corrFourier (folded): sign and the (2 - omega_1) factor of q^corr
    "qcorr_sign": ("0.5 * (2.0 - omega1) * Pres * corr_flux",
                   "-0.5 * (2.0 - omega1) * Pres * corr_flux"),
    "qcorr_factor": ("0.5 * (2.0 - omega1) * Pres * corr_flux",
                     "0.5 * (2.0 - omega) * Pres * corr_flux"),
    "qcorr_dropped": ("0.5 * (2.0 - omega1) * Pres * corr_flux", "0.0 * Pres * corr_flux"),
    # Eq. qdiff (folded): the factor omega_1 of the interdiffusion flux
    "qdiff_factor": ("omega1 * rho * diff_flux", "omega * rho * diff_flux"),
    "qdiff_half": ("omega1 * rho * diff_flux", "0.5 * omega1 * rho * diff_flux"),
    "qdiff_dropped": ("omega1 * rho * diff_flux", "0.0 * rho * diff_flux"),
}


def mutation(name):
    old, new = MUTATIONS[name]
    return mutated_oracle(old, new)
