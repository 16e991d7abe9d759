"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every computation runs in the CUDA library _lib/libpaper2108lbm.so; this
module only converts arrays, structs and status codes.  If the library has
not been built, importing raises: there is no CPU fallback.

Functions carry the C names (lbm_create, lbm_init_fields, lbm_step,
lbm_moments, lbm_destroy, ...).  ``Solver`` is a small convenience wrapper
that owns one handle.  Device memory comes from PyTorch's caching allocator
(through the allocation hooks of lbm_config) and the default stream is
torch's current stream.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_SPECIES = 9
MAX_REACTIONS = 32
NCP = 3

LBM_D2Q9, LBM_D3Q27 = 0, 1
LBM_FP64, LBM_FP32_STORE, LBM_FP16_OFFSET = 0, 1, 2
LBM_PERIODIC, LBM_BOUNCE_BACK, LBM_TMS_WALL, LBM_INLET, LBM_OUTLET = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_ERR_INVALID", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
                4: "LBM_ERR_NEWTON", 5: "LBM_ERR_NONFINITE", 6: "LBM_ERR_RANGE",
                7: "LBM_ERR_TIMEOUT", 8: "LBM_ERR_STATE"}
FACE_KINDS = {"periodic": LBM_PERIODIC, "bounce_back": LBM_BOUNCE_BACK,
              "tms": LBM_TMS_WALL, "inlet": LBM_INLET, "outlet": LBM_OUTLET}
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32_STORE, "fp16": LBM_FP16_OFFSET}
# the fixed scratch array of lbm_step_noalloc (LBM_NOALLOC_MAX_NODES x 61
# fields + 32 doubles), resident on every GPU that loads the library
NOALLOC_MAX_NODES = 16384
NOALLOC_SCRATCH_BYTES = (NOALLOC_MAX_NODES * 61 + 32) * 8


class lbm_mechanism(C.Structure):
    _fields_ = [
        ("n_species", C.c_int), ("n_reactions", C.c_int),
        ("molar_mass", C.c_double * MAX_SPECIES),
        ("cp", (C.c_double * NCP) * MAX_SPECIES),
        ("h_formation", C.c_double * MAX_SPECIES),
        ("s_standard", C.c_double * MAX_SPECIES),
        ("nu_f", (C.c_int * MAX_SPECIES) * MAX_REACTIONS),
        ("nu_r", (C.c_int * MAX_SPECIES) * MAX_REACTIONS),
        ("arrhenius", (C.c_double * 3) * MAX_REACTIONS),
        ("third_body", C.c_int * MAX_REACTIONS),
        ("efficiency", (C.c_double * MAX_SPECIES) * MAX_REACTIONS),
        ("reversible", C.c_int * MAX_REACTIONS),
        ("D0", (C.c_double * MAX_SPECIES) * MAX_SPECIES),
        ("D_T_exponent", C.c_double), ("mu0", C.c_double),
        ("mu_T_exponent", C.c_double), ("prandtl", C.c_double),
        ("viscosity_model", C.c_int), ("mu0_species", C.c_double * MAX_SPECIES),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_config(C.Structure):
    _fields_ = [
        ("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("precision", C.c_int), ("substeps", C.c_int), ("dx", C.c_double),
        ("c_ref", C.c_double), ("T_max", C.c_double), ("mech", lbm_mechanism),
        ("face_bc", C.c_int * 6), ("wall_T", C.c_double * 6),
        ("solid_mask", C.POINTER(C.c_uint8)), ("solid_bc", C.c_int),
        ("wall_T_nodes", C.POINTER(C.c_double)),
        ("inlet_u", C.POINTER(C.c_double)), ("inlet_u_uniform", C.c_double * 3),
        ("inlet_Y", C.c_double * MAX_SPECIES), ("inlet_T", C.c_double),
        ("inlet_P", C.c_double), ("outlet_P", C.c_double), ("outlet_sigma", C.c_double),
        ("newton_max_iter", C.c_int), ("newton_rtol", C.c_double),
        ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", C.c_void_p),
        ("stream", C.c_void_p), ("device", C.c_int), ("inlet_simplified", C.c_int),
        ("wall_dist", C.POINTER(C.c_double)), ("wall_normal", C.POINTER(C.c_double)),
        ("outlet_length", C.c_double), ("chem_fp64", C.c_int),
    ]


class lbm_launch(C.Structure):
    _fields_ = [("chem_lanes", C.c_int), ("collide_split", C.c_int), ("persistent", C.c_int),
                ("nodes_per_thread", C.c_int)]


class lbm_diag(C.Structure):
    _fields_ = [("hrr_integral", C.c_double), ("hrr_max", C.c_double),
                ("flame_x", C.c_double), ("T_max", C.c_double), ("u_max", C.c_double)]


class lbm_info(C.Structure):
    _fields_ = [("Q", C.c_int), ("D", C.c_int), ("L", C.c_int), ("M", C.c_int),
                ("n_nodes", C.c_longlong), ("c_ref", C.c_double), ("dt", C.c_double),
                ("dx", C.c_double), ("bytes_per_population", C.c_size_t),
                ("device_bytes", C.c_size_t), ("steps_done", C.c_longlong)]


EXPORTS = {
    # name: (restype, argtypes)
    "lbm_config_defaults": (None, [C.POINTER(lbm_config)]),
    "lbm_bytes_required": (C.c_size_t, [C.POINTER(lbm_config)]),
    "lbm_create": (C.c_int, [C.POINTER(lbm_config), C.POINTER(C.c_void_p)]),
    "lbm_init_fields": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "lbm_init_fields_pressure": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "lbm_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_step_timed": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int]),
    "lbm_batch_step": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int]),
    "lbm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_void_p)]),
    "lbm_batch_run": (C.c_int, [C.c_void_p, C.c_int]),
    "lbm_batch_destroy": (C.c_int, [C.c_void_p]),
    "lbm_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(lbm_launch)]),
    "lbm_ff_check": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p]),
    "lbm_exp64_check": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p]),
    "lbm_batch_set_launch": (C.c_int, [C.c_void_p, C.POINTER(lbm_launch)]),
    "lbm_batch_get_launch": (C.c_int, [C.c_void_p, C.POINTER(lbm_launch)]),
    "lbm_set_launch": (C.c_int, [C.c_void_p, C.POINTER(lbm_launch)]),
    "lbm_get_launch": (C.c_int, [C.c_void_p, C.POINTER(lbm_launch)]),
    "lbm_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(lbm_launch)]),
    "lbm_moments": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int]),
    "lbm_get_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "lbm_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(lbm_diag)]),
    "lbm_diagnostics_planes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(lbm_diag)]),
    "lbm_synchronize": (C.c_int, [C.c_void_p]),
    "lbm_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_size_t)]),
    "lbm_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lbm_get_info": (C.c_int, [C.c_void_p, C.POINTER(lbm_info)]),
    "lbm_destroy": (C.c_int, [C.c_void_p]),
    "lbm_last_error": (C.c_char_p, [C.c_void_p]),
    "lbm_fma_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "lbm_wait_probe": (C.c_int, [C.c_int, C.c_longlong, C.POINTER(C.c_longlong)]),
    "lbm_worklist": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                               C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lbm_get_planes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "lbm_set_planes": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "lbm_step_noalloc": (C.c_int, [C.POINTER(lbm_config), C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.POINTER(C.c_char_p)]),
}

_lib = None


def library_path():
    return _build.LIBPATH


def load_library():
    """Load the built library (never builds; run build.build() first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library {path} is missing: build it with "
            "`python -m paper_2108_07605_gb300.build` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status, handle=None):
    if status != 0:
        msg = load_library().lbm_last_error(handle)
        raise LBMError(status, msg.decode() if msg else "")


def mechanism_struct(mech):
    """Marshal a mechanism table (lbm_workloads.mechanism.Mechanism or any
    object with the same attributes) into lbm_mechanism."""
    s = lbm_mechanism()
    M, R = mech.n_species, mech.n_reactions
    if M > MAX_SPECIES or R > MAX_REACTIONS:
        raise ValueError("mechanism exceeds the library limits")
    s.n_species, s.n_reactions = M, R
    for a in range(M):
        s.molar_mass[a] = float(mech.molar_mass[a])
        for k in range(NCP):
            s.cp[a][k] = float(mech.cp_coeffs[a][k])
        s.h_formation[a] = float(mech.h_formation[a])
        s.s_standard[a] = float(mech.s_standard[a])
        for b in range(M):
            s.D0[a][b] = float(mech.D0[a][b])
    for r in range(R):
        for a in range(M):
            s.nu_f[r][a] = int(mech.nu_f[r][a])
            s.nu_r[r][a] = int(mech.nu_r[r][a])
            s.efficiency[r][a] = float(mech.efficiency[r][a])
        for k in range(3):
            s.arrhenius[r][k] = float(mech.arrhenius[r][k])
        s.third_body[r] = int(mech.third_body[r])
        s.reversible[r] = int(mech.reversible[r])
    s.D_T_exponent = float(mech.D_T_exponent)
    s.mu0 = float(mech.mu0)
    s.mu_T_exponent = float(mech.mu_T_exponent)
    s.prandtl = float(mech.prandtl)
    s.viscosity_model = 1 if getattr(mech, "viscosity_model", "mixture") == "wilke" else 0
    mu_sp = getattr(mech, "mu0_species", None)
    if mu_sp is not None:
        for a, v in enumerate(np.asarray(mu_sp, dtype=np.float64)):
            s.mu0_species[a] = float(v)
    return s


# ---- same-name wrappers of the C entry points ---------------------------------
def lbm_config_defaults():
    cfg = lbm_config()
    load_library().lbm_config_defaults(C.byref(cfg))
    return cfg


def lbm_bytes_required(cfg):
    return int(load_library().lbm_bytes_required(C.byref(cfg)))


def lbm_create(cfg):
    h = C.c_void_p()
    st = load_library().lbm_create(C.byref(cfg), C.byref(h))
    _check(st, None)
    return h


def _ptr(arr):
    """(pointer, on_device) of a host numpy array or a CUDA torch tensor."""
    if arr is None:
        return None, 0
    if hasattr(arr, "data_ptr"):
        if not arr.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if arr.is_cuda:
            return C.c_void_p(arr.data_ptr()), 1
        return C.c_void_p(arr.data_ptr()), 0
    if not (isinstance(arr, np.ndarray) and arr.flags["C_CONTIGUOUS"]):
        raise ValueError("host arrays must be C-contiguous numpy arrays")
    return arr.ctypes.data_as(C.c_void_p), 0


def _same_side(*arrs):
    sides = {_ptr(a)[1] for a in arrs if a is not None}
    if len(sides) > 1:
        raise ValueError("mix of host and device arrays")
    return sides.pop() if sides else 0


def lbm_init_fields(h, rho, u, T, Y):
    on = _same_side(rho, u, T, Y)
    _check(load_library().lbm_init_fields(h, _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0],
                                          _ptr(Y)[0], on), h)


def lbm_init_fields_pressure(h, P, u, T, Y):
    on = _same_side(P, u, T, Y)
    _check(load_library().lbm_init_fields_pressure(h, _ptr(P)[0], _ptr(u)[0], _ptr(T)[0],
                                                   _ptr(Y)[0], on), h)


def lbm_step(h, nsteps):
    _check(load_library().lbm_step(h, int(nsteps)), h)


def lbm_batch_step(handles, nsteps):
    """Advance several handles together (one launch per kernel per step)."""
    hs = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                       for h in handles])
    _check(load_library().lbm_batch_step(hs, len(handles), int(nsteps)), hs[0])


class BatchPlan:
    """lbm_batch_t with the handles it was made for (errors of the plan's calls
    are reported on its first handle)."""

    def __init__(self, ptr, handles):
        self._as_parameter_ = ptr
        self.handles = handles


def lbm_batch_create(handles):
    """Capture a batch plan (CUDA graphs of the batched step) for handles."""
    hs = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h
                                       for h in handles])
    out = C.c_void_p()
    _check(load_library().lbm_batch_create(hs, len(handles), C.byref(out)), hs[0])
    return BatchPlan(out, list(hs))


def lbm_batch_run(plan, nsteps):
    _check(load_library().lbm_batch_run(plan, int(nsteps)), plan.handles[0])


def lbm_batch_destroy(plan):
    _check(load_library().lbm_batch_destroy(plan), plan.handles[0])


def _launch_dict(l):
    return {"chem_lanes": l.chem_lanes, "collide_split": l.collide_split,
            "persistent": l.persistent, "nodes_per_thread": l.nodes_per_thread}


def lbm_batch_autotune(plan, trial_steps=3):
    """Returns the chosen placement {"chem_lanes": 1/4/8, "collide_split": 0/1}."""
    out = lbm_launch()
    _check(load_library().lbm_batch_autotune(plan, int(trial_steps), C.byref(out)),
           plan.handles[0])
    return _launch_dict(out)


def lbm_exp64_check(x):
    """The library's FP64 exp (reaction rates) at the points x (1-D float64)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.empty_like(x)
    _check(load_library().lbm_exp64_check(x.ctypes.data, x.size, e.ctypes.data))
    return e


def lbm_ff_check(x):
    """Float-float exp and log of the library at the points x (1-D float64):
    returns (exp, log) as float64 arrays (hi + lo of each result)."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.empty_like(x)
    lg = np.empty_like(x)
    _check(load_library().lbm_ff_check(x.ctypes.data, x.size, e.ctypes.data, lg.ctypes.data))
    return e, lg


def lbm_batch_set_launch(plan, chem_lanes=-1, collide_split=-1, persistent=-1,
                         nodes_per_thread=-1):
    l = lbm_launch(chem_lanes=int(chem_lanes), collide_split=int(collide_split),
                   persistent=int(persistent), nodes_per_thread=int(nodes_per_thread))
    _check(load_library().lbm_batch_set_launch(plan, C.byref(l)), plan.handles[0])


def lbm_batch_get_launch(plan):
    out = lbm_launch()
    _check(load_library().lbm_batch_get_launch(plan, C.byref(out)), plan.handles[0])
    return _launch_dict(out)


def lbm_set_launch(h, chem_lanes=-1, collide_split=-1, persistent=-1, nodes_per_thread=-1):
    l = lbm_launch(chem_lanes=int(chem_lanes), collide_split=int(collide_split),
                   persistent=int(persistent), nodes_per_thread=int(nodes_per_thread))
    _check(load_library().lbm_set_launch(h, C.byref(l)), h)


def lbm_get_launch(h):
    out = lbm_launch()
    _check(load_library().lbm_get_launch(h, C.byref(out)), h)
    return _launch_dict(out)


def lbm_autotune(h, trial_steps=3):
    out = lbm_launch()
    _check(load_library().lbm_autotune(h, int(trial_steps), C.byref(out)), h)
    return _launch_dict(out)


def lbm_step_timed(h, nsteps, kernel_ms=None):
    """Returns per-kernel device milliseconds [moments, collision] (added to
    kernel_ms when given)."""
    arr = (C.c_double * 2)(*(kernel_ms or (0.0, 0.0)))
    _check(load_library().lbm_step_timed(h, int(nsteps), arr, 2), h)
    return [arr[0], arr[1]]


def lbm_moments(h, rho=None, u=None, T=None, Y=None, E=None):
    on = _same_side(rho, u, T, Y, E)
    _check(load_library().lbm_moments(h, _ptr(rho)[0], _ptr(u)[0], _ptr(T)[0],
                                      _ptr(Y)[0], _ptr(E)[0], on), h)


def lbm_diagnostics(h):
    out = lbm_diag()
    _check(load_library().lbm_diagnostics(h, C.byref(out)), h)
    return {k: getattr(out, k) for k, _ in lbm_diag._fields_}


def lbm_diagnostics_planes(h, x0, nplanes):
    """lbm_diagnostics over the planes x0 .. x0 + nplanes - 1 only."""
    out = lbm_diag()
    _check(load_library().lbm_diagnostics_planes(h, int(x0), int(nplanes), C.byref(out)), h)
    return {k: getattr(out, k) for k, _ in lbm_diag._fields_}


def lbm_get_populations(h, out):
    p, on = _ptr(out)
    _check(load_library().lbm_get_populations(h, p, on), h)


def lbm_synchronize(h):
    _check(load_library().lbm_synchronize(h), h)


def lbm_get_state(h):
    n = C.c_size_t(0)
    _check(load_library().lbm_get_state(h, None, C.byref(n)), h)
    buf = np.empty(n.value, dtype=np.uint8)
    _check(load_library().lbm_get_state(h, buf.ctypes.data_as(C.c_void_p), C.byref(n)), h)
    return buf


def lbm_set_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().lbm_set_state(h, buf.ctypes.data_as(C.c_void_p), buf.size), h)


def lbm_get_info(h):
    info = lbm_info()
    _check(load_library().lbm_get_info(h, C.byref(info)), h)
    return info


def lbm_destroy(h):
    _check(load_library().lbm_destroy(h), None)


def _noalloc_buffer(name, t, dtype, count, device):
    """The C function cannot see its buffers' sizes, so they are checked
    here: a contiguous CUDA tensor on `device` of `dtype` with at least
    `count` elements."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the config names cuda:{device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements, the grid needs {count}")


def lbm_step_noalloc(cfg, pops_in, pops_out, T_guess):
    """One step on caller-owned device buffers with no device allocation
    (for callers that cannot allocate; see include/lbm.h)."""
    import torch
    D = 3 if cfg.lattice == LBM_D3Q27 else 2
    Q = 27 if D == 3 else 9
    N = int(cfg.nx) * int(cfg.ny) * int(cfg.nz)
    L = int(cfg.mech.n_species) + 1
    store = {LBM_FP64: torch.float64, LBM_FP32_STORE: torch.float32,
             LBM_FP16_OFFSET: torch.float16}.get(int(cfg.precision))
    if store is None:
        raise ValueError(f"unknown precision {cfg.precision}")
    _noalloc_buffer("pops_in", pops_in, store, L * Q * N, int(cfg.device))
    _noalloc_buffer("pops_out", pops_out, store, L * Q * N, int(cfg.device))
    _noalloc_buffer("T_guess", T_guess, torch.float64, N, int(cfg.device))
    err = C.c_char_p()
    st = load_library().lbm_step_noalloc(C.byref(cfg), _ptr(pops_in)[0], _ptr(pops_out)[0],
                                         _ptr(T_guess)[0], C.byref(err))
    if st != 0:
        raise LBMError(st, err.value.decode() if err.value else "")


def lbm_get_planes(h, x0, nplanes, buf):
    """Copy planes x0 .. x0+nplanes-1 (populations in the storage precision,
    then the temperature guesses) into buf (a numpy array or a CUDA tensor
    of at least the plane bytes, any dtype)."""
    p, on = _ptr(buf)
    _check(load_library().lbm_get_planes(h, int(x0), int(nplanes), p, on), h)


def lbm_set_planes(h, x0, nplanes, buf):
    """Copy buf (as written by lbm_get_planes) into planes x0 .. x0+nplanes-1."""
    p, on = _ptr(buf)
    _check(load_library().lbm_set_planes(h, int(x0), int(nplanes), p, on), h)


def lbm_fma_peak(fp64):
    """Measured FMA throughput (TFLOP/s) of the current device, FP64 or FP32."""
    out = C.c_double(0.0)
    _check(load_library().lbm_fma_peak(1 if fp64 else 0, C.byref(out)))
    return out.value


def lbm_worklist(nodes, n_if, nodes_per_thread=1, collide_split=1):
    """The single-launch step's work-list for domains of the given node and
    interface-node counts (host only): returns (items [n, 5] int64: kind,
    domain, first, dep, flag; the number of sync words)."""
    import numpy as np
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    n_if = np.ascontiguousarray(n_if, dtype=np.int64)
    lib = load_library()
    cnt, ns = C.c_int(0), C.c_int(0)
    _check(lib.lbm_worklist(nodes.ctypes.data, n_if.ctypes.data, nodes.size,
                            int(nodes_per_thread), int(collide_split), None, 0,
                            C.byref(cnt), C.byref(ns)))
    items = np.zeros((max(cnt.value, 1), 5), dtype=np.int64)
    _check(lib.lbm_worklist(nodes.ctypes.data, n_if.ctypes.data, nodes.size,
                            int(nodes_per_thread), int(collide_split), items.ctypes.data,
                            cnt.value, C.byref(cnt), C.byref(ns)))
    return items[:cnt.value], ns.value


def lbm_wait_probe(set_word, timeout_ns):
    """The bounded device wait of the single-launch batched step on a word
    that is set (set_word) or that nothing sets: returns (saw_word, abort,
    microseconds)."""
    out = (C.c_longlong * 3)()
    _check(load_library().lbm_wait_probe(1 if set_word else 0, int(timeout_ns), out))
    return int(out[0]), int(out[1]), int(out[2])


def lbm_last_error(h=None):
    msg = load_library().lbm_last_error(h)
    return msg.decode() if msg else ""


# ---- torch-backed allocation hooks -------------------------------------------------
class _TorchAllocator:
    """Allocation hooks that draw from torch's caching allocator on `device`."""

    def __init__(self, device, stream_ptr):
        import torch
        self._torch = torch
        self.device = device
        self.stream_ptr = stream_ptr

        def alloc(nbytes, user):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                          self.stream_ptr)
            except Exception:
                return None

        def free(ptr, user):
            torch.cuda.caching_allocator_delete(ptr)

        self.alloc = ALLOC_FN(alloc)
        self.free = FREE_FN(free)


def make_config(mech, lattice="D3Q27", shape=(16, 16, 16), dx=1e-3, precision="fp64",
                substeps=2, c_ref=0.0, T_max=3000.0, faces=None, newton_max_iter=50,
                newton_rtol=1e-13, device=0, stream=None, use_torch_allocator=True,
                wall_T=None, solid=None, solid_kind="tms", inlet=None, outlet=None,
                chem_fp64=0, wall_dist=None, wall_normal=None):
    """Build an lbm_config from Python values.  Returns (cfg, keepalive).

    wall_T: scalar (every TMS face) or a grid array [nz, ny, nx] (per node);
    solid: optional grid array of solid nodes; inlet: dict(u, T, Y, P) with u
    a 3-vector or a [3, nz, ny, nx] array (m/s); outlet: dict(P, sigma);
    chem_fp64: with precision "fp32", the temperature solve and chemistry in
    native FP64 instead of float-float; wall_dist [nz, ny, nx] and
    wall_normal [3, nz, ny, nx] (together): off-grid TMS targets."""
    cfg = lbm_config_defaults()
    cfg.lattice = LBM_D3Q27 if lattice == "D3Q27" else LBM_D2Q9
    cfg.nx, cfg.ny, cfg.nz = (int(v) for v in shape)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.chem_fp64 = int(chem_fp64)
    cfg.substeps = int(substeps)
    cfg.dx = float(dx)
    cfg.c_ref = float(c_ref)
    cfg.T_max = float(T_max)
    cfg.mech = mechanism_struct(mech)
    for f, kind in enumerate(faces or ("periodic",) * 6):
        cfg.face_bc[f] = FACE_KINDS[kind] if isinstance(kind, str) else int(kind)
    cfg.newton_max_iter = int(newton_max_iter)
    cfg.newton_rtol = float(newton_rtol)
    cfg.device = int(device)
    keep = []
    if wall_T is not None:
        wt = np.asarray(wall_T, dtype=np.float64)
        if wt.ndim == 0:
            for f in range(6):
                cfg.wall_T[f] = float(wt)
        else:
            wt = np.ascontiguousarray(wt.reshape(-1))
            keep.append(wt)
            cfg.wall_T_nodes = wt.ctypes.data_as(C.POINTER(C.c_double))
    if (wall_dist is None) != (wall_normal is None):
        raise ValueError("wall_dist and wall_normal go together")
    if wall_dist is not None:
        wd = np.ascontiguousarray(np.asarray(wall_dist, dtype=np.float64).reshape(-1))
        wn = np.ascontiguousarray(np.asarray(wall_normal, dtype=np.float64).reshape(-1))
        if wd.size != cfg.nx * cfg.ny * cfg.nz or wn.size != 3 * wd.size:
            raise ValueError("wall_dist needs one value per node and wall_normal three")
        keep += [wd, wn]
        cfg.wall_dist = wd.ctypes.data_as(C.POINTER(C.c_double))
        cfg.wall_normal = wn.ctypes.data_as(C.POINTER(C.c_double))
    if solid is not None:
        sm = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8).reshape(-1))
        keep.append(sm)
        cfg.solid_mask = sm.ctypes.data_as(C.POINTER(C.c_uint8))
        cfg.solid_bc = FACE_KINDS[solid_kind] if isinstance(solid_kind, str) else int(solid_kind)
    if inlet is not None:
        u = np.asarray(inlet["u"], dtype=np.float64)
        if u.ndim == 1:
            for d in range(3):
                cfg.inlet_u_uniform[d] = float(u[d])
        else:
            uu = np.ascontiguousarray(u.reshape(-1))
            keep.append(uu)
            cfg.inlet_u = uu.ctypes.data_as(C.POINTER(C.c_double))
        cfg.inlet_T = float(inlet["T"])
        cfg.inlet_P = float(inlet.get("P", 101325.0))
        cfg.inlet_simplified = 1 if inlet.get("simplified", False) else 0
        for a, y in enumerate(np.asarray(inlet["Y"], dtype=np.float64)):
            cfg.inlet_Y[a] = float(y)
    if outlet is not None:
        cfg.outlet_P = float(outlet.get("P", 101325.0))
        cfg.outlet_sigma = float(outlet.get("sigma", 0.25))
        cfg.outlet_length = float(outlet.get("length") or 0.0)
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream(device).cuda_stream
        except Exception:
            stream = None
    cfg.stream = C.c_void_p(stream) if stream else None
    if use_torch_allocator:
        alloc = _TorchAllocator(device, stream or 0)
        cfg.dev_alloc = alloc.alloc
        cfg.dev_free = alloc.free
        keep.append(alloc)
    return cfg, keep


class Solver:
    """One lbm_t handle with numpy/torch-friendly methods."""

    def __init__(self, mech, **kw):
        self.mech = mech
        self.cfg, self._keep = make_config(mech, **kw)
        self.h = lbm_create(self.cfg)
        self.info = lbm_get_info(self.h)
        self.N = int(self.info.n_nodes)
        self.M = int(self.info.M)

    def init_fields(self, rho, u, T, Y):
        lbm_init_fields(self.h, *[_flat(a) for a in (rho, u, T, Y)])

    def init_fields_pressure(self, P, u, T, Y):
        lbm_init_fields_pressure(self.h, *[_flat(a) for a in (P, u, T, Y)])

    def step(self, n=1):
        lbm_step(self.h, n)

    def set_launch(self, chem_lanes=-1, collide_split=-1, persistent=-1, nodes_per_thread=-1):
        lbm_set_launch(self.h, chem_lanes, collide_split, persistent, nodes_per_thread)

    def launch(self):
        return lbm_get_launch(self.h)

    def autotune(self, trial_steps=3):
        return lbm_autotune(self.h, trial_steps)

    def moments(self):
        N, M = self.N, self.M
        out = dict(rho=np.empty(N), u=np.empty(3 * N), T=np.empty(N), Y=np.empty(M * N),
                   E=np.empty(N))
        lbm_moments(self.h, out["rho"], out["u"], out["T"], out["Y"], out["E"])
        out["u"] = out["u"].reshape(3, N)
        out["Y"] = out["Y"].reshape(M, N)
        return out

    def diagnostics(self):
        return lbm_diagnostics(self.h)

    def populations(self):
        info = self.info
        out = np.empty(info.L * info.Q * self.N)
        lbm_get_populations(self.h, out)
        return out.reshape(info.L, info.Q, self.N)

    def synchronize(self):
        lbm_synchronize(self.h)

    def get_state(self):
        return lbm_get_state(self.h)

    def set_state(self, buf):
        lbm_set_state(self.h, buf)

    def close(self):
        if self.h is not None:
            h, self.h = self.h, None
            lbm_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _flat(a):
    if hasattr(a, "data_ptr"):
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
