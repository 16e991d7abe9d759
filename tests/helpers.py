"""Shared test plumbing: run one workload through the CPU oracle and through
the CUDA library (via the C-ABI binding) on identical seeded inputs."""
import numpy as np

from lbm_workloads.mechanism import h2_air_synthetic
from oracle import OracleLBM, thermo


def perturbed_box(shape, lattice="D3Q27", seed=7, T0=1400.0, dx=1e-3, mech=None,
                  amp_T=2e-2, amp_u=3.0, amp_Y=2e-3):
    """A periodic box with seeded temperature, velocity and composition
    perturbations, so that gradients, diffusion velocities and the energy
    flux corrections are all exercised."""
    from lbm_workloads import fields
    from lbm_workloads.mechanism import air_mole_fractions, mole_to_mass_fractions
    mech = mech or h2_air_synthetic()
    nx, ny, nz = shape
    rng = fields.philox(seed)
    g = (nz, ny, nx)
    M = mech.n_species
    if "H2" in mech.species:
        Y0 = mole_to_mass_fractions(mech, air_mole_fractions(mech, 0.5))
    else:
        Y0 = np.full(M, 1.0 / M)
    w = dict(dx=dx, T_max=3000.0, substeps=2, faces=("periodic",) * 6, seed=seed)
    Y = np.empty((M,) + g)
    noise = rng.uniform(-1.0, 1.0, size=(M,) + g)
    for a in range(M):
        Y[a] = Y0[a] * (1.0 + amp_Y * noise[a]) + amp_Y * 1e-3 * (noise[a] + 1.0)
    Y /= Y.sum(axis=0, keepdims=True)
    u = amp_u * rng.uniform(-1.0, 1.0, size=(3,) + g)
    if lattice == "D2Q9":
        u[2] = 0.0
    T = T0 * (1.0 + amp_T * rng.uniform(-1.0, 1.0, size=g))
    P = np.full(g, 101325.0) * (1.0 + 1e-3 * rng.uniform(-1.0, 1.0, size=g))
    w.update(shape=shape, lattice=lattice, P=P, T=T, u=u, Y=Y,
             name=f"perturbed box {shape} {lattice}")
    return w


def make_oracle(mech, w, c_ref=0.0):
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], c_ref=c_ref,
                  T_max=w["T_max"], substeps=w["substeps"])
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    return o


def make_gpu(mech, w, precision="fp64", c_ref=0.0):
    from paper_2108_07605_gb300 import lbm
    s = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                   precision=precision, substeps=w["substeps"], c_ref=c_ref,
                   T_max=w["T_max"])
    s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    return s


def oracle_populations(o):
    L, Q = o.pops.shape[:2]
    return o.pops.reshape(L, Q, -1)


def max_rel_err_per_lattice(got, ref):
    """max |got - ref| / max |ref| for each lattice."""
    L = ref.shape[0]
    out = np.empty(L)
    for l in range(L):
        scale = np.max(np.abs(ref[l]))
        out[l] = np.max(np.abs(got[l] - ref[l])) / scale
    return out
