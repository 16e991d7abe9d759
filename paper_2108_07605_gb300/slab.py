"""X-slab domain decomposition of the reactive LBM step (host logic).

The paper runs one domain.  Every quantity a node's step needs comes from
the node and its neighbours: the pull streaming reads the post-collision
populations one plane away (Sec. 4.1 Eq. advection), and the isotropic
gradients of the collision (Sec. 3.4, last paragraph) read the moments of
the streamed state one plane away again.  A node's new populations therefore
depend on the previous post-collision state at most HALO = 2 planes away
(the boundary procedures of Sec. 4 read the node itself and the outlet's
upstream neighbour, one plane away).  So a slab of planes [x_lo, x_hi) that
holds, besides its own planes, copies of its neighbours' two nearest planes
(and their temperature guesses, the Newton starting points) advances its own
planes exactly as the undivided domain does, provided the copies are
refreshed before every step.  The copies' own updates are discarded.

Layout: the global x extent is split into contiguous slabs, one per rank.
A slab's local domain is its planes plus HALO ghost planes on every side
that has a neighbouring slab (both sides when x is periodic, neither at a
non-periodic global face, which keeps its boundary condition).  Internal
faces are periodic in the local domain: the ghost planes wrap onto each
other there, and what they compute is overwritten by the next exchange.

Exchange: before each step every slab sends its first and last HALO planes
to the neighbouring slabs' ghost planes (point-to-point, torch.distributed
P2P over gloo or NCCL, or direct copies between handles in one process).
Nothing here computes a step of the method: the engine (the CUDA library's
handle, or any object with get_planes / set_planes / step) does.

Diagnostics: each slab evaluates the flame diagnostics of its own planes
(engine.diagnostics), and one all-gather of five scalars per slab combines
them into those of the whole domain (heat release integrals add, maxima
take the largest, the flame position follows the largest heat release).
"""
import numpy as np

HALO = 2

# per-node arrays of a workload (lbm_workloads.fields): x is the last axis
_NODE_FIELDS = ("P", "T", "u", "Y", "wall_T", "solid", "wall_dist", "wall_normal")


class SlabLayout:
    """Partition of nx planes into `world` slabs; periodic_x: whether the
    global -x / +x faces are periodic (then every slab has two neighbours)."""

    def __init__(self, nx, world, periodic_x):
        if world < 1 or nx < world * HALO:
            raise ValueError(f"{nx} planes cannot form {world} slabs of >= {HALO} planes")
        self.nx, self.world, self.periodic = int(nx), int(world), bool(periodic_x)
        base, extra = divmod(self.nx, self.world)
        self.bounds = []
        x = 0
        for r in range(self.world):
            w = base + (1 if r < extra else 0)
            self.bounds.append((x, x + w))
            x += w

    def neighbours(self, rank):
        """(left, right) ranks, None where the slab ends at a global face."""
        if self.world == 1:
            return None, None
        left = rank - 1 if rank > 0 else (self.world - 1 if self.periodic else None)
        right = rank + 1 if rank < self.world - 1 else (0 if self.periodic else None)
        return left, right

    def local(self, rank):
        """(x_lo, x_hi, g_lo, g_hi): the slab's own planes [x_lo, x_hi) and its
        local domain [g_lo, g_hi) in global x (g_lo < 0 or g_hi > nx wrap)."""
        x_lo, x_hi = self.bounds[rank]
        left, right = self.neighbours(rank)
        return (x_lo, x_hi, x_lo - (HALO if left is not None else 0),
                x_hi + (HALO if right is not None else 0))


def slab_workload(w, layout, rank):
    """The workload of one slab: every per-node array restricted to the
    slab's local domain (wrapping in x where it is periodic), the grid
    shape, and the x faces: internal faces periodic, global faces kept."""
    x_lo, x_hi, g_lo, g_hi = layout.local(rank)
    left, right = layout.neighbours(rank)
    cols = np.arange(g_lo, g_hi) % layout.nx
    out = dict(w)
    for k in _NODE_FIELDS:
        if k in w and w[k] is not None and np.ndim(w[k]) >= 3:
            out[k] = np.ascontiguousarray(np.asarray(w[k])[..., cols])
    nx, ny, nz = w["shape"]
    out["shape"] = (g_hi - g_lo, ny, nz)
    faces = list(w.get("faces", ("periodic",) * 6))
    if left is not None:
        faces[0] = "periodic"
    if right is not None:
        faces[1] = "periodic"
    out["faces"] = tuple(faces)
    if w.get("outlet") is not None:
        # the LODI outlet's length stays the whole domain's
        out["outlet"] = dict(w["outlet"], length=float(nx))
    if w.get("inlet") is not None:
        inlet = dict(w["inlet"])
        u = np.asarray(inlet["u"])
        if u.ndim > 1:
            inlet["u"] = np.ascontiguousarray(u[..., cols])
        out["inlet"] = inlet
    out["slab"] = dict(rank=rank, x_lo=x_lo, x_hi=x_hi, g_lo=g_lo, g_hi=g_hi)
    return out


class Exchange:
    """Halo exchange of one slab.  engine: get_planes(x0, n) -> buffer (a
    tensor), set_planes(x0, n, buffer); pg: torch.distributed (or None for
    one slab).  Planes are in local x."""

    def __init__(self, layout, rank, pg=None):
        self.layout, self.rank, self.pg = layout, rank, pg
        x_lo, x_hi, g_lo, g_hi = layout.local(rank)
        self.own = (x_lo - g_lo, x_hi - g_lo)          # local [first, last) own plane
        self.left, self.right = layout.neighbours(rank)

    def exchange(self, engine):
        """Send the first HALO own planes to the left neighbour's right ghosts
        and the last HALO own planes to the right neighbour's left ghosts;
        receive this slab's ghosts.  Tags keep the two directions apart when
        both neighbours are the same rank."""
        if self.left is None and self.right is None:
            return
        dist = self.pg
        a, b = self.own
        ops, recv = [], []
        TO_LEFT, TO_RIGHT = 1, 2
        if self.left is not None:
            send = engine.get_planes(a, HALO)
            buf = engine.empty_planes(HALO)
            ops.append(dist.P2POp(dist.isend, send, self.left, tag=TO_LEFT))
            ops.append(dist.P2POp(dist.irecv, buf, self.left, tag=TO_RIGHT))
            recv.append((a - HALO, buf))
        if self.right is not None:
            send = engine.get_planes(b - HALO, HALO)
            buf = engine.empty_planes(HALO)
            ops.append(dist.P2POp(dist.isend, send, self.right, tag=TO_RIGHT))
            ops.append(dist.P2POp(dist.irecv, buf, self.right, tag=TO_LEFT))
            recv.append((b, buf))
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        for x0, buf in recv:
            engine.set_planes(x0, HALO, buf)

    def step(self, engine, nsteps=1):
        for _ in range(nsteps):
            self.exchange(engine)
            engine.step(1)


def combine_diagnostics(parts):
    """Flame diagnostics of the whole domain from those of the slabs' own
    planes (each a dict of lbm_diagnostics_planes with flame_x already in
    global x): heat release integrals add, maxima take the largest, the flame
    position is that of the largest heat release (among equal maxima the
    smallest x, as on one domain: the slabs are in x order)."""
    out = {"hrr_integral": float(sum(p["hrr_integral"] for p in parts))}
    best = None
    for p in parts:
        if best is None or p["hrr_max"] > best["hrr_max"]:
            best = p
    out["hrr_max"] = best["hrr_max"]
    out["flame_x"] = best["flame_x"]
    out["T_max"] = max(p["T_max"] for p in parts)
    out["u_max"] = max(p["u_max"] for p in parts)
    return out


def own_diagnostics(layout, rank, engine, dx):
    """The flame diagnostics of the slab's own planes (engine.diagnostics(x0,
    n), x in the slab's local grid), the flame position shifted to global x
    (the local plane i is the global plane g_lo + i)."""
    x_lo, x_hi, g_lo, g_hi = layout.local(rank)
    own = engine.diagnostics(x_lo - g_lo, x_hi - x_lo)
    fx = own["flame_x"]
    if fx == fx:   # not NaN: the plane index times dx, as on one domain
        fx = (int(round(fx / dx)) + g_lo) * dx
    return dict(own, flame_x=fx)


def diagnostics(layout, rank, engine, dx, pg=None):
    """The whole domain's flame diagnostics from every rank's slab: each rank
    evaluates its own planes (own_diagnostics), and one all-gather of five
    scalars per rank (torch.distributed, or none for one slab) combines them
    identically on every rank."""
    own = own_diagnostics(layout, rank, engine, dx)
    if pg is None or layout.world == 1:
        return combine_diagnostics([own])
    import torch
    keys = ("hrr_integral", "hrr_max", "flame_x", "T_max", "u_max")
    mine = torch.tensor([float(own[k]) for k in keys], dtype=torch.float64)
    if pg.get_backend() == "nccl":
        mine = mine.cuda()
    gathered = [torch.empty_like(mine) for _ in range(layout.world)]
    pg.all_gather(gathered, mine)
    parts = [dict(zip(keys, g.cpu().tolist())) for g in gathered]
    return combine_diagnostics(parts)


def exchange_in_process(layout, engines):
    """The same exchange between slabs held by one process (engines[rank]):
    direct copies, no collective."""
    grabbed = []
    for r, eng in enumerate(engines):
        x_lo, x_hi, g_lo, g_hi = layout.local(r)
        a, b = x_lo - g_lo, x_hi - g_lo
        left, right = layout.neighbours(r)
        if left is not None:
            grabbed.append((left, "right", eng.get_planes(a, HALO)))
        if right is not None:
            grabbed.append((right, "left", eng.get_planes(b - HALO, HALO)))
    for dst, side, buf in grabbed:
        x_lo, x_hi, g_lo, g_hi = layout.local(dst)
        x0 = (x_hi - g_lo) if side == "right" else 0
        engines[dst].set_planes(x0, HALO, buf)


class SolverEngine:
    """Engine adapter for an lbm.Solver: halo planes as byte tensors on the
    solver's GPU (device-to-device copies through lbm_get_planes /
    lbm_set_planes)."""

    def __init__(self, solver):
        import torch
        from . import lbm
        self.s, self.lbm, self.torch = solver, lbm, torch
        info = solver.info
        nx, ny, nz = solver.cfg.nx, solver.cfg.ny, solver.cfg.nz
        self.plane_bytes = ny * nz * (info.L * info.Q * info.bytes_per_population + 8)

    def empty_planes(self, n):
        return self.torch.empty(n * self.plane_bytes, dtype=self.torch.uint8,
                                device=f"cuda:{self.s.cfg.device}")

    def get_planes(self, x0, n):
        buf = self.empty_planes(n)
        self.lbm.lbm_get_planes(self.s.h, x0, n, buf)
        return buf

    def set_planes(self, x0, n, buf):
        self.lbm.lbm_set_planes(self.s.h, x0, n, buf)

    def step(self, n=1):
        self.s.step(n)

    def diagnostics(self, x0, n):
        return self.lbm.lbm_diagnostics_planes(self.s.h, x0, n)
