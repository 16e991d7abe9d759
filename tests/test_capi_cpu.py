"""The C-ABI library without a GPU: it builds, loads, exports every entry
point include/lbm.h declares, its struct layout matches the binding's, and
the host-only paths (defaults, validation, byte counts) behave as documented.
No compute call is made here."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from lbm_workloads.mechanism import h2_air_synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lbm():
    from paper_2108_07605_gb300 import build
    build.build()
    from paper_2108_07605_gb300 import lbm as binding
    binding.load_library()
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lbm):
    names = declared_functions()
    assert "lbm_create" in names and "lbm_step" in names and "lbm_destroy" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lbm.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    for n in names:
        assert n in lbm.EXPORTS
        assert callable(getattr(lbm, n))


def test_struct_layout_matches_c(lbm, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lbm_mechanism),
         sizeof(lbm_config), sizeof(lbm_info), offsetof(lbm_config, mech),
         offsetof(lbm_config, face_bc), offsetof(lbm_config, inlet_u),
         offsetof(lbm_config, dev_alloc), offsetof(lbm_config, stream),
         offsetof(lbm_mechanism, D0), offsetof(lbm_config, solid_mask),
         offsetof(lbm_config, wall_T_nodes), offsetof(lbm_config, inlet_simplified),
         sizeof(lbm_launch), sizeof(lbm_diag));
  return 0;
}}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    got = [C.sizeof(lbm.lbm_mechanism), C.sizeof(lbm.lbm_config), C.sizeof(lbm.lbm_info),
           lbm.lbm_config.mech.offset, lbm.lbm_config.face_bc.offset,
           lbm.lbm_config.inlet_u.offset, lbm.lbm_config.dev_alloc.offset,
           lbm.lbm_config.stream.offset, lbm.lbm_mechanism.D0.offset,
           lbm.lbm_config.solid_mask.offset, lbm.lbm_config.wall_T_nodes.offset,
           lbm.lbm_config.inlet_simplified.offset, C.sizeof(lbm.lbm_launch),
           C.sizeof(lbm.lbm_diag)]
    assert got == vals


def test_defaults_and_bytes_required(lbm):
    cfg = lbm.lbm_config_defaults()
    assert cfg.substeps == 2 and cfg.newton_max_iter == 50 and cfg.newton_rtol == 1e-13
    assert cfg.lattice == lbm.LBM_D3Q27 and cfg.precision == lbm.LBM_FP64
    # zeroed mechanism is invalid -> 0 bytes
    assert lbm.lbm_bytes_required(cfg) == 0
    cfg.mech = lbm.mechanism_struct(h2_air_synthetic())
    cfg.nx, cfg.ny, cfg.nz = 16, 16, 16
    n = lbm.lbm_bytes_required(cfg)
    N, L, Q = 16 ** 3, 10, 27
    assert n >= 2 * L * Q * N * 8
    cfg.precision = lbm.LBM_FP32_STORE
    n32 = lbm.lbm_bytes_required(cfg)
    NF = 61                       # moment-record fields of D3Q27 with 9 species
    # collision-parameter fields (split collision): theta_b, V_b, rho_b (M, M*D, M),
    # cF, 2 beta, drho (M-1 each), u, P^ex, W (D each), rho, omega, U, theta
    NP = 9 + 27 + 9 + 3 * 8 + 3 * 3 + 4
    assert n - n32 == (2 * L * Q + NF + NP) * N * 4   # populations and scratch halve


@pytest.mark.parametrize("mutate, text", [
    (lambda c: setattr(c, "nx", 0), "grid"),
    (lambda c: setattr(c, "substeps", 0), "substeps"),
    (lambda c: setattr(c, "dx", -1.0), "dx"),
    (lambda c: setattr(c.mech, "n_species", 5), "n_species"),
    (lambda c: setattr(c, "lattice", 7), "lattice"),
    (lambda c: setattr(c, "newton_max_iter", 0), "Newton"),
])
def test_invalid_configs_rejected_before_any_device_call(lbm, mutate, text):
    cfg, keep = lbm.make_config(h2_air_synthetic(), shape=(4, 4, 4),
                                use_torch_allocator=False, stream=0)
    mutate(cfg)
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(cfg)
    assert e.value.status == 1
    assert text.lower() in str(e.value).lower()


def test_null_handle_calls_fail_cleanly(lbm):
    lib = lbm.load_library()
    assert lib.lbm_step(None, 1) == 1
    assert lib.lbm_synchronize(None) == 1
    assert lib.lbm_destroy(None) == 0
    assert "NULL" in lbm.lbm_last_error(None)


def test_mechanism_marshalling_round_trip(lbm):
    mech = h2_air_synthetic()
    s = lbm.mechanism_struct(mech)
    assert s.n_species == 9 and s.n_reactions == 21
    assert np.isclose(s.molar_mass[8], mech.molar_mass[8])
    assert s.nu_f[4][0] == 1 and s.nu_r[4][3] == 2          # H2 + M <=> 2 H + M
    assert s.third_body[4] == 1 and s.efficiency[4][2] == 12.0


def _check_worklist(items, nsync, nodes, nif, npt, split):
    """The single launch's list: stage order, coverage, and every dependency
    on items earlier in the list (what lets its bounded waits end)."""
    stage = {0: 1, 1: 1, 2: 2, 4: 2, 3: 3}
    kinds = items[:, 0]
    st = np.array([stage[int(k)] for k in kinds])
    assert np.all(np.diff(st) >= 0)
    tile = 128 * npt
    n = len(nodes)
    n1 = [int(np.sum((kinds <= 1) & (items[:, 1] == d))) for d in range(n)]
    flag_at = {}
    for i, (kind, dom, first, dep, flag) in enumerate(items):
        if kind == 2:
            flag_at[int(flag)] = (i, int(dom), int(first))
    for d in range(n):
        mine = items[items[:, 1] == d]
        bnd = mine[mine[:, 0] == 0][:, 2]
        assert list(bnd) == list(range(0, nif[d], 128))
        for kind, step in ((1, tile), (2 if split else 4, tile), (3, 32)):
            if kind == 3 and not split:
                continue
            firsts = mine[mine[:, 0] == kind][:, 2]
            assert list(firsts) == list(range(0, nodes[d], step)), (d, kind)
    for i, (kind, dom, first, dep, flag) in enumerate(items):
        if kind in (2, 4):
            assert dep == n1[dom]
            before = items[:i]
            assert np.sum((before[:, 0] <= 1) & (before[:, 1] == dom)) == n1[dom]
        elif kind == 3:
            j, pdom, pfirst = flag_at[int(dep)]
            assert j < i and pdom == dom and pfirst <= first < pfirst + tile
    nprep = int(np.sum(kinds == 2))
    assert nsync == 2 + n + nprep
    assert sorted(flag_at) == list(range(nprep))


@pytest.mark.parametrize("npt,split", [(1, 1), (2, 1), (4, 1), (1, 0), (4, 0)])
def test_single_launch_worklist_order(lbm, npt, split):
    nodes = [4096, 130, 96000, 1, 300]
    nif = [0, 40, 14400, 1, 300]
    items, nsync = lbm.lbm_worklist(nodes, nif, npt, split)
    _check_worklist(items, nsync, nodes, nif, npt, split)
    with pytest.raises(lbm.LBMError):
        lbm.lbm_worklist([10], [11], npt, split)          # more interface nodes than nodes
    with pytest.raises(lbm.LBMError):
        lbm.lbm_worklist([10], [0], 3, split)             # nodes per thread
