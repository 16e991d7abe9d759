"""The x-slab domain decomposition (paper_2108_07605_gb300/slab.py) on the
CPU: two gloo ranks, each advancing one slab of the domain with the CPU
oracle as the engine and exchanging two halo planes (populations and
temperature guesses) with its neighbour before every step, reproduce the
undivided oracle run exactly on the slabs' own planes: a periodic box (a
neighbour on both sides, the same rank), the flame layout (inlet and LODI
outlet at the global faces) and the staircase tube with off-grid TMS
targets.  The ranks' flame diagnostics, each of its own planes and combined
by one all-gather, equal the undivided domain's.  The layout arithmetic is
checked without ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2108_07605_gb300 import slab

HALO = slab.HALO


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(name):
    from lbm_workloads import fields
    from lbm_workloads.mechanism import h2_air_synthetic
    mech = h2_air_synthetic()
    if name == "box":
        w = fields.perturbed_box((12, 5, 4), "D3Q27", mech=mech)
    elif name == "flame":
        w = fields.flame_1d(seed=3, nx=24, ny=3, nz=2, x_ign=6, mech=mech)
    else:
        w = fields.microtube(nx=16, ny=9, nz=9, radius=3.6, mech=mech, offgrid=True)
    return mech, w


class OracleEngine:
    """The oracle as a slab engine: halo planes as float64 tensors; flame
    diagnostics of a range of planes from the oracle's moments."""

    def __init__(self, o, mech=None, w=None):
        import torch
        self.o, self.torch = o, torch
        self.mech, self.w = mech, w
        L, Q, nz, ny, _ = o.pops.shape
        self.per_plane = L * Q * nz * ny + nz * ny

    def empty_planes(self, n):
        return self.torch.empty(n * self.per_plane, dtype=self.torch.float64)

    def get_planes(self, x0, n):
        p = self.o.pops[..., x0:x0 + n].reshape(-1)
        t = self.o.T[..., x0:x0 + n].reshape(-1)
        return self.torch.from_numpy(np.concatenate([p, t]))

    def set_planes(self, x0, n, buf):
        a = buf.numpy()
        shp = self.o.pops[..., x0:x0 + n].shape
        k = int(np.prod(shp))
        self.o.pops[..., x0:x0 + n] = a[:k].reshape(shp)
        self.o.T[..., x0:x0 + n] = a[k:].reshape(self.o.T[..., x0:x0 + n].shape)

    def step(self, n=1):
        self.o.step(n)

    def diagnostics(self, x0, n):
        from oracle import diagnostics
        mo = self.o.moments()
        sl = (Ellipsis, slice(x0, x0 + n))
        solid = self.w.get("solid")
        fluid = None if solid is None else ~np.asarray(solid)[sl]
        d = diagnostics.diagnostics(self.mech, mo["rho"][sl], mo["u"][sl], mo["T"][sl],
                                    mo["Y"][sl], self.w["dx"], 3, n, fluid)
        d["flame_x"] += x0 * self.w["dx"]          # x in this engine's grid
        return d


def _rank_main(rank, world, port, name, nsteps, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from helpers import make_oracle
    mech, w = _case(name)
    layout = slab.SlabLayout(w["shape"][0], world, w["faces"][0] == "periodic")
    wl = slab_workload = slab.slab_workload(w, layout, rank)
    eng = OracleEngine(make_oracle(mech, wl), mech, wl)
    ex = slab.Exchange(layout, rank, dist)
    ex.step(eng, nsteps)
    a, b = ex.own
    diag = slab.diagnostics(layout, rank, eng, w["dx"], dist)
    out[rank] = (wl["slab"]["x_lo"], eng.o.pops[..., a:b].copy(), eng.o.T[..., a:b].copy(), diag)
    del slab_workload
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name,nsteps", [("box", 4), ("flame", 5), ("tube", 3)])
def test_two_gloo_slabs_equal_the_undivided_domain(name, nsteps):
    from helpers import make_oracle
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, name, nsteps, out), nprocs=2, join=True)
        res = dict(out)
    mech, w = _case(name)
    o = make_oracle(mech, w)
    o.step(nsteps)
    # the whole domain's flame diagnostics, combined by the ranks' all-gather
    dref = OracleEngine(o, mech, w).diagnostics(0, w["shape"][0])
    for rank in (0, 1):
        d = res[rank][3]
        assert d["hrr_integral"] == pytest.approx(dref["hrr_integral"], rel=1e-12)
        for k in ("hrr_max", "flame_x", "T_max", "u_max"):
            assert d[k] == dref[k], (rank, k)
    for rank in (0, 1):
        x_lo, pops, T, _ = res[rank]
        n = pops.shape[-1]
        ref = o.pops[..., x_lo:x_lo + n]
        fluid = slice(None)
        if w.get("solid") is not None:
            keep = ~np.asarray(w["solid"])[..., x_lo:x_lo + n]
            assert np.array_equal(pops[:, :, keep], ref[:, :, keep]), rank
        else:
            assert np.array_equal(pops[fluid], ref[fluid]), rank
        assert np.allclose(T, o.T[..., x_lo:x_lo + n], rtol=1e-12, atol=0), rank


def test_layout_and_workload_slicing():
    lay = slab.SlabLayout(25, 3, periodic_x=False)
    assert lay.bounds == [(0, 9), (9, 17), (17, 25)]
    assert lay.neighbours(0) == (None, 1) and lay.neighbours(2) == (1, None)
    assert lay.local(0) == (0, 9, 0, 9 + HALO)
    assert lay.local(1) == (9, 17, 9 - HALO, 17 + HALO)
    per = slab.SlabLayout(12, 2, periodic_x=True)
    assert per.neighbours(0) == (1, 1)
    assert per.local(0) == (0, 6, -HALO, 6 + HALO)
    mech, w = _case("flame")
    wl = slab.slab_workload(w, slab.SlabLayout(24, 2, False), 1)
    assert wl["shape"] == (12 + HALO, 3, 2)
    assert wl["faces"][0] == "periodic" and wl["faces"][1] == "outlet"
    assert np.array_equal(wl["T"], w["T"][..., 12 - HALO:])
    with pytest.raises(ValueError):
        slab.SlabLayout(3, 2, False)
