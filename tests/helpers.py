"""Shared test plumbing: run one workload through the CPU oracle and through
the CUDA library (via the C-ABI binding) on identical seeded inputs."""
import numpy as np

from lbm_workloads.mechanism import h2_air_synthetic
from lbm_workloads.fields import perturbed_box  # noqa: F401
from oracle import OracleLBM, thermo


BC_KEYS = ("faces", "inlet", "outlet", "wall_T", "solid", "solid_kind", "wall_dist",
           "wall_normal")


def boundary_spec(w):
    """The workload's boundary description, or None for a periodic box."""
    faces = w.get("faces", ("periodic",) * 6)
    if all(f == "periodic" for f in faces) and w.get("solid") is None:
        return None
    return {k: w[k] for k in BC_KEYS if k in w}


def make_oracle(mech, w, c_ref=0.0):
    o = OracleLBM(mech, w["lattice"], w["shape"], w["dx"], c_ref=c_ref,
                  T_max=w["T_max"], substeps=w["substeps"], boundaries=boundary_spec(w))
    rho = thermo.density_from_pressure(mech, w["P"], w["T"], w["Y"])
    o.init_fields(rho, w["u"], w["T"], w["Y"])
    return o


def make_gpu(mech, w, precision="fp64", c_ref=0.0):
    """precision: "fp64", "fp32" (float-float chemistry), "fp32c64" (FP32
    storage with the temperature solve and chemistry in FP64) or "fp16"."""
    from paper_2108_07605_gb300 import lbm
    bc = boundary_spec(w) or {}
    chem64 = precision == "fp32c64"
    s = lbm.Solver(mech, lattice=w["lattice"], shape=w["shape"], dx=w["dx"],
                   precision="fp32" if chem64 else precision, chem_fp64=int(chem64),
                   substeps=w["substeps"], c_ref=c_ref, T_max=w["T_max"], **bc)
    s.init_fields_pressure(w["P"], w["u"], w["T"], w["Y"])
    return s


def oracle_populations(o):
    L, Q = o.pops.shape[:2]
    return o.pops.reshape(L, Q, -1)


def max_rel_err_per_lattice(got, ref, mask=None):
    """max |got - ref| / max |ref| for each lattice; `mask` (flat, True =
    compare) excludes solid nodes, whose populations are not defined."""
    L = ref.shape[0]
    if mask is not None:
        got, ref = got[:, :, mask], ref[:, :, mask]
    out = np.empty(L)
    for l in range(L):
        scale = np.max(np.abs(ref[l]))
        out[l] = np.max(np.abs(got[l] - ref[l])) / scale
    return out
