"""Shared test plumbing: run one workload through the CPU oracle and through
the CUDA library (via the C-ABI binding) on identical seeded inputs."""
import numpy as np

from lbm_workloads.mechanism import h2_air_synthetic
from lbm_workloads.fields import perturbed_box  # noqa: F401
from oracle import OracleLBM, thermo


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
