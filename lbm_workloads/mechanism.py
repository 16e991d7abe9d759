"""Synthetic mechanism tables: species, thermodynamics, reactions, transport.

This module is input data only.  It holds no step of the lattice Boltzmann
method; the CUDA library and the CPU oracle each evaluate thermodynamics,
rates and transport from these numbers with their own code.

The paper (Sec. 3.6, "Coupling between lattice Boltzmann and chemical
kinetics") takes thermodynamic data, Arrhenius rates and transport
coefficients of the nine-species hydrogen/air mechanism of Li et al. (2004)
from Cantera.  Neither that mechanism file nor Cantera is available to this
project, and the table is NOT recreated from memory.  ``h2_air_synthetic()``
is a synthetic, hydrogen/air-shaped stand-in written for this project:

* the nine species of the paper, with molar masses built from element masses;
* standard formation enthalpies and entropies at T0 = 298.15 K rounded to
  textbook thermochemistry values (physical constants, not mechanism data);
* heat capacities c_p/R_U = a0 + a1 T + a2 T^2, round synthetic coefficients
  giving plausible magnitudes between 300 K and 3500 K;
* 21 reversible elementary reactions with the reaction structure typical of
  H2/O2 chemistry (chain branching, recombination with third bodies, HO2 and
  H2O2 channels) and ROUND SYNTHETIC Arrhenius constants; reverse rates
  follow from equilibrium constants of this table's own thermodynamics, so
  detailed balance holds by construction;
* a power-law transport model: binary diffusion D_ab(T, P) =
  D0_ab (T/T0)^1.75 (P0/P), viscosity mu = mu0 (T/T0)^0.7, conductivity
  lambda = mu c_p / Pr.

Units are SI throughout: kg/mol, J/mol, J/(mol K), m^3/mol, s, Pa, m^2/s.
Arrhenius: k = A T^b exp(-Ea / (R_U T)); for a reaction of total molecular
order n (third body counted), A has units (m^3/mol)^(n-1) / s.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

R_UNIVERSAL = 8.314462618      # J/(mol K)
T_STANDARD = 298.15            # K, reference temperature T0 of Sec. 3.6
P_STANDARD = 101325.0          # Pa, reference pressure P0 of Sec. 3.6

MAX_SPECIES = 9
MAX_REACTIONS = 32
N_CP = 3                       # c_p/R_U = a0 + a1 T + a2 T^2

ELEMENT_MASS = {"H": 1.008e-3, "O": 15.999e-3, "N": 14.007e-3}   # kg/mol


@dataclass
class Mechanism:
    """A species/reaction/transport table.  Arrays are indexed [species] or
    [reaction, species]; the last species is the one the lattice slaves."""
    species: List[str]
    elements: List[str]
    composition: np.ndarray        # [M, n_elements] atoms per molecule
    molar_mass: np.ndarray         # [M] kg/mol
    cp_coeffs: np.ndarray          # [M, N_CP] c_p/R_U polynomial in T (K)
    h_formation: np.ndarray        # [M] J/mol at T0
    s_standard: np.ndarray         # [M] J/(mol K) at T0, P0
    nu_f: np.ndarray               # [R, M] reactant stoichiometric coefficients
    nu_r: np.ndarray               # [R, M] product stoichiometric coefficients
    arrhenius: np.ndarray          # [R, 3] (A, b, Ea)
    third_body: np.ndarray         # [R] 1 if a third body M participates
    efficiency: np.ndarray         # [R, M] third-body efficiencies
    reversible: np.ndarray         # [R] 1 if the reverse rate is included
    D0: np.ndarray                 # [M, M] binary diffusion at T0, P0 (m^2/s)
    D_T_exponent: float = 1.75
    mu0: float = 1.8e-5            # Pa s at T0
    mu_T_exponent: float = 0.7
    prandtl: float = 0.7
    # per-species viscosities at T0 (Pa s) for the Wilke mixing rule; the
    # model in use: "mixture" (mu0 power law) or "wilke"
    mu0_species: np.ndarray = None
    viscosity_model: str = "mixture"
    label: str = ""
    equations: List[str] = field(default_factory=list)

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return int(self.nu_f.shape[0])

    def index(self, name: str) -> int:
        return self.species.index(name)


def _molar_masses(composition, elements):
    em = np.array([ELEMENT_MASS[e] for e in elements])
    return composition @ em


# Species order of the build: the majority-mass inert N2 is last (slaved).
_H2AIR_SPECIES = ["H2", "O2", "H2O", "H", "O", "OH", "HO2", "H2O2", "N2"]
_H2AIR_ELEMENTS = ["H", "O", "N"]
_H2AIR_COMPOSITION = {
    "H2": (2, 0, 0), "O2": (0, 2, 0), "H2O": (2, 1, 0), "H": (1, 0, 0),
    "O": (0, 1, 0), "OH": (1, 1, 0), "HO2": (1, 2, 0), "H2O2": (2, 2, 0),
    "N2": (0, 0, 2),
}
# c_p/R_U = a0 + a1 T + a2 T^2 (synthetic, round coefficients)
_H2AIR_CP = {
    "H2": (3.40, 2.0e-4, 3.0e-8),
    "O2": (3.30, 8.0e-4, -1.5e-7),
    "H2O": (3.70, 1.2e-3, -1.0e-7),
    "H": (2.50, 0.0, 0.0),
    "O": (2.60, -5.0e-5, 0.0),
    "OH": (3.45, 3.0e-4, 3.0e-8),
    "HO2": (3.80, 1.6e-3, -2.5e-7),
    "H2O2": (4.90, 2.0e-3, -3.0e-7),
    "N2": (3.25, 6.0e-4, -1.0e-7),
}
# standard formation enthalpy (J/mol) and entropy (J/(mol K)) at 298.15 K,
# rounded textbook thermochemistry values
_H2AIR_HF = {"H2": 0.0, "O2": 0.0, "H2O": -241826.0, "H": 217999.0,
             "O": 249175.0, "OH": 37300.0, "HO2": 12020.0, "H2O2": -135880.0,
             "N2": 0.0}
_H2AIR_S0 = {"H2": 130.68, "O2": 205.15, "H2O": 188.83, "H": 114.72,
             "O": 161.06, "OH": 183.74, "HO2": 229.0, "H2O2": 232.99,
             "N2": 191.61}
# collision diameters (Angstrom, rounded) for the synthetic diffusion table
_H2AIR_SIGMA = {"H2": 2.9, "O2": 3.5, "H2O": 2.6, "H": 2.0, "O": 2.75,
                "OH": 2.75, "HO2": 3.45, "H2O2": 3.45, "N2": 3.6}

_TB_DEFAULT = {"H2": 2.5, "H2O": 12.0}
# (reactants, products, A, b, Ea[J/mol], third-body efficiencies or None)
_H2AIR_REACTIONS: List[Tuple[dict, dict, float, float, float, object]] = [
    ({"H": 1, "O2": 1}, {"O": 1, "OH": 1}, 1.0e10, -0.5, 70.0e3, None),
    ({"O": 1, "H2": 1}, {"H": 1, "OH": 1}, 5.0e-2, 2.7, 26.0e3, None),
    ({"OH": 1, "H2": 1}, {"H": 1, "H2O": 1}, 2.0e2, 1.5, 14.0e3, None),
    ({"O": 1, "H2O": 1}, {"OH": 2}, 3.0e0, 2.0, 56.0e3, None),
    ({"H2": 1}, {"H": 2}, 5.0e13, -1.5, 436.0e3, _TB_DEFAULT),
    ({"O": 2}, {"O2": 1}, 6.0e3, -0.5, 0.0, _TB_DEFAULT),
    ({"O": 1, "H": 1}, {"OH": 1}, 5.0e6, -1.0, 0.0, _TB_DEFAULT),
    ({"H": 1, "OH": 1}, {"H2O": 1}, 4.0e10, -2.0, 0.0, _TB_DEFAULT),
    ({"H": 1, "O2": 1}, {"HO2": 1}, 5.0e8, -1.5, 0.0,
     {"H2": 2.0, "H2O": 11.0, "O2": 0.8}),
    ({"HO2": 1, "H": 1}, {"H2": 1, "O2": 1}, 2.0e7, 0.0, 3.0e3, None),
    ({"HO2": 1, "H": 1}, {"OH": 2}, 7.0e7, 0.0, 1.0e3, None),
    ({"HO2": 1, "O": 1}, {"O2": 1, "OH": 1}, 3.0e7, 0.0, 0.0, None),
    ({"HO2": 1, "OH": 1}, {"H2O": 1, "O2": 1}, 3.0e7, 0.0, -2.0e3, None),
    ({"HO2": 2}, {"H2O2": 1, "O2": 1}, 4.0e8, 0.0, 50.0e3, None),
    ({"HO2": 2}, {"H2O2": 1, "O2": 1}, 1.0e5, 0.0, -7.0e3, None),
    ({"H2O2": 1}, {"OH": 2}, 1.0e11, 0.0, 190.0e3, _TB_DEFAULT),
    ({"H2O2": 1, "H": 1}, {"H2O": 1, "OH": 1}, 2.0e7, 0.0, 17.0e3, None),
    ({"H2O2": 1, "H": 1}, {"HO2": 1, "H2": 1}, 5.0e7, 0.0, 33.0e3, None),
    ({"H2O2": 1, "O": 1}, {"OH": 1, "HO2": 1}, 1.0e1, 2.0, 17.0e3, None),
    ({"H2O2": 1, "OH": 1}, {"HO2": 1, "H2O": 1}, 1.0e6, 0.0, 0.0, None),
    ({"H2O2": 1, "OH": 1}, {"HO2": 1, "H2O": 1}, 6.0e8, 0.0, 40.0e3, None),
]


def _equation(reac, prod, tb):
    def side(d):
        s = " + ".join((f"{n} {k}" if n > 1 else k) for k, n in d.items())
        return s + (" + M" if tb is not None else "")
    return f"{side(reac)} <=> {side(prod)}"


def _binary_diffusion_table(species, molar_mass, sigma, d_ref=2.0e-5,
                            ref="N2"):
    """Synthetic D0_ab at (T0, P0): kinetic-theory scaling
    D ~ sqrt(1/m_a + 1/m_b) / sigma_ab^2, normalised so D0(ref, ref) = d_ref."""
    M = len(species)
    mr = molar_mass[species.index(ref)]
    sr = sigma[species.index(ref)]
    D = np.zeros((M, M))
    for a in range(M):
        for b in range(M):
            mass = np.sqrt((1.0 / molar_mass[a] + 1.0 / molar_mass[b]) / (2.0 / mr))
            sab = 0.5 * (sigma[a] + sigma[b])
            D[a, b] = d_ref * mass * (sr / sab) ** 2
    return D


def _species_viscosities(species, molar_mass, sigma, mu_ref=1.78e-5, ref="N2"):
    """Synthetic species viscosities at T0 by kinetic-theory scaling
    mu ~ sqrt(m) / sigma^2, normalised so mu(ref) = mu_ref."""
    mr = molar_mass[species.index(ref)]
    sr = sigma[species.index(ref)]
    return mu_ref * np.sqrt(molar_mass / mr) * (sr / sigma) ** 2


def with_viscosity_model(mech: Mechanism, model: str) -> Mechanism:
    """A copy of mech with the viscosity model set ("mixture" or "wilke")."""
    import dataclasses
    if model not in ("mixture", "wilke"):
        raise ValueError(model)
    if model == "wilke" and mech.mu0_species is None:
        raise ValueError("the mechanism has no species viscosities")
    return dataclasses.replace(mech, viscosity_model=model)


def h2_air_synthetic() -> Mechanism:
    """Synthetic 9-species / 21-reaction H2/air-shaped mechanism (see module
    docstring).  N2 is last, so it is the slaved species."""
    sp = list(_H2AIR_SPECIES)
    M, R = len(sp), len(_H2AIR_REACTIONS)
    comp = np.array([_H2AIR_COMPOSITION[s] for s in sp], dtype=float)
    mm = _molar_masses(comp, _H2AIR_ELEMENTS)
    cp = np.array([_H2AIR_CP[s] for s in sp], dtype=float)
    hf = np.array([_H2AIR_HF[s] for s in sp])
    s0 = np.array([_H2AIR_S0[s] for s in sp])
    nu_f = np.zeros((R, M))
    nu_r = np.zeros((R, M))
    arr = np.zeros((R, 3))
    tb = np.zeros(R, dtype=np.int32)
    eff = np.ones((R, M))
    eqs = []
    for r, (reac, prod, A, b, Ea, effs) in enumerate(_H2AIR_REACTIONS):
        for k, n in reac.items():
            nu_f[r, sp.index(k)] += n
        for k, n in prod.items():
            nu_r[r, sp.index(k)] += n
        arr[r] = (A, b, Ea)
        if effs is not None:
            tb[r] = 1
            for k, e in effs.items():
                eff[r, sp.index(k)] = e
        eqs.append(_equation(reac, prod, effs))
    sigma = np.array([_H2AIR_SIGMA[s] for s in sp])
    D0 = _binary_diffusion_table(sp, mm, sigma)
    return Mechanism(species=sp, elements=list(_H2AIR_ELEMENTS),
                     composition=comp, molar_mass=mm, cp_coeffs=cp,
                     h_formation=hf, s_standard=s0, nu_f=nu_f, nu_r=nu_r,
                     arrhenius=arr, third_body=tb, efficiency=eff,
                     reversible=np.ones(R, dtype=np.int32), D0=D0,
                     mu0_species=_species_viscosities(sp, mm, sigma),
                     label="synthetic H2/air-shaped, 9 species, 21 reactions",
                     equations=eqs)


def binary_inert(molar_mass=28.0e-3, D0=2.0e-5, cp_over_R=3.5,
                 mu0=1.8e-5, h_formation=(0.0, 0.0)) -> Mechanism:
    """Two non-reacting species "A" and "B" of equal molar mass and constant
    heat capacity: the binary-diffusion and single-fluid test cases (Sec. 2.1
    limit of the Stefan-Maxwell model).  By default chemically identical;
    h_formation (J/mol) gives them different formation enthalpies, so that
    interdiffusion carries enthalpy."""
    sp = ["A", "B"]
    comp = np.array([[1.0], [1.0]])
    return Mechanism(
        species=sp, elements=["X"], composition=comp,
        molar_mass=np.array([molar_mass, molar_mass]),
        cp_coeffs=np.array([[cp_over_R, 0.0, 0.0], [cp_over_R, 0.0, 0.0]]),
        h_formation=np.array([float(h) for h in h_formation]),
        s_standard=np.array([150.0, 150.0]),
        nu_f=np.zeros((0, 2)), nu_r=np.zeros((0, 2)), arrhenius=np.zeros((0, 3)),
        third_body=np.zeros(0, dtype=np.int32), efficiency=np.ones((0, 2)),
        reversible=np.zeros(0, dtype=np.int32),
        D0=np.full((2, 2), D0), mu0=mu0, mu0_species=np.array([mu0, mu0]),
        label="binary inert, equal masses")


def air_mole_fractions(mech: Mechanism, phi: float) -> np.ndarray:
    """Fresh H2/air mole fractions at equivalence ratio phi, air = O2 + 3.76 N2
    by moles (H2 : O2 = 2 phi : 1)."""
    X = np.zeros(mech.n_species)
    X[mech.index("H2")] = 2.0 * phi
    X[mech.index("O2")] = 1.0
    X[mech.index("N2")] = 3.76
    return X / X.sum()


def mole_to_mass_fractions(mech: Mechanism, X: np.ndarray) -> np.ndarray:
    w = X * mech.molar_mass
    return w / w.sum()
