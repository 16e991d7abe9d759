"""Seeded synthetic workloads: grids, boundary layouts and initial fields.

Input generation only: these functions draw random numbers and lay out
arrays; they contain no step of the lattice Boltzmann method.  Both the CUDA
library (through its Python binding) and the CPU oracle take their inputs
from here.  Random draws use numpy's Philox counter-based generator keyed by
the seed, so the same bits reach both sides.

Every workload is a dict:
  lattice      "D3Q27" or "D2Q9"
  shape        (nx, ny, nz)
  dx           lattice spacing (m)
  T_max        temperature bound for the default reference speed (K)
  substeps     reaction sub-steps l
  faces        boundary kind per face (-x, +x, -y, +y, -z, +z)
  P, T         [nz, ny, nx] initial pressure (Pa) and temperature (K)
  u            [3, nz, ny, nx] initial velocity (m/s)
  Y            [M, nz, ny, nx] initial mass fractions
  steps        nominal number of steps of the workload
and, where the faces need them, the inlet and wall data.
"""
import numpy as np

from .mechanism import (P_STANDARD, air_mole_fractions, mole_to_mass_fractions,
                        h2_air_synthetic)


def philox(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def _uniform_fields(mech, shape, T, P, Y, u=(0.0, 0.0, 0.0)):
    nx, ny, nz = shape
    g = (nz, ny, nx)
    return dict(
        P=np.full(g, float(P)), T=np.full(g, float(T)),
        u=np.stack([np.full(g, float(v)) for v in u]),
        Y=np.stack([np.full(g, float(y)) for y in Y]))


def reactor(seed=0, n=16, phi=0.5, T0=1200.0, P=P_STANDARD, dx=1.0e-3,
            perturbation=1e-3, steps=200, mech=None):
    """Homogeneous constant-volume reactor: n^3 periodic D3Q27 box, fresh
    H2/air at equivalence ratio phi, zero velocity, T = T0 (1 + eps U(-1,1))
    with a seeded uniform perturbation (the paper's perfectly stirred reactor,
    Sec. 3.8, on a larger box)."""
    mech = mech or h2_air_synthetic()
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, phi))
    w = _uniform_fields(mech, (n, n, n), T0, P, Y)
    if perturbation:
        w["T"] = T0 * (1.0 + perturbation * philox(seed).uniform(-1.0, 1.0, size=w["T"].shape))
    w.update(lattice="D3Q27", shape=(n, n, n), dx=dx, T_max=3000.0, substeps=2,
             faces=("periodic",) * 6, steps=steps, name=f"reactor {n}^3 D3Q27 phi={phi}",
             seed=seed)
    return w


def flame_1d(seed=0, nx=1024, ny=4, nz=4, phi=0.5, T_u=300.0, T_b=1500.0,
             x_ign=256, width=4.0, dx=12.5e-6, steps=20000, mech=None):
    """Quasi-1D premixed flame: nx x ny x nz D3Q27, periodic in y and z,
    velocity inlet at x = 0 (fresh mixture at phi, T_u, speed u_in drawn from
    the seed in [0.5, 2] m/s) and pressure outlet at x = nx-1; a tanh
    temperature kernel T_u -> T_b centred at x_ign ignites the mixture."""
    mech = mech or h2_air_synthetic()
    rng = philox(seed)
    u_in = float(rng.uniform(0.5, 2.0))
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, phi))
    w = _uniform_fields(mech, (nx, ny, nz), T_u, P_STANDARD, Y, u=(u_in, 0.0, 0.0))
    x = np.arange(nx, dtype=float)
    Tx = T_u + (T_b - T_u) * 0.5 * (1.0 + np.tanh((x - x_ign) / width))
    w["T"] = np.broadcast_to(Tx, (nz, ny, nx)).copy()
    w.update(lattice="D3Q27", shape=(nx, ny, nz), dx=dx, T_max=3000.0, substeps=2,
             faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"),
             inlet=dict(u=np.array([u_in, 0.0, 0.0]), T=T_u, Y=Y, P=P_STANDARD),
             outlet=dict(P=P_STANDARD), steps=steps, seed=seed,
             name=f"flame {nx}x{ny}x{nz} D3Q27 phi={phi} u_in={u_in:.3f}")
    return w


def shear_wave(nx=32, ny=1, nz=1, amplitude=1e-3, background=0.0, T=300.0,
               dx=1e-6, lattice="D3Q27", mech=None):
    """Decaying transverse shear wave u_y(x) = amplitude sin(2 pi x/nx) in a
    uniform single-fluid (binary, equal composition) state, periodic box."""
    from .mechanism import binary_inert
    mech = mech or binary_inert()
    nzz = nz if lattice == "D3Q27" else 1
    w = _uniform_fields(mech, (nx, ny, nzz), T, P_STANDARD, (0.5, 0.5))
    x = np.arange(nx)
    w["u"][1] = amplitude * np.sin(2.0 * np.pi * x / nx)[None, None, :]
    w["u"][0] = background
    w.update(lattice=lattice, shape=(nx, ny, nzz), dx=dx, T_max=T, substeps=1,
             faces=("periodic",) * 6, steps=0, name="shear wave")
    return w


def perturbed_box(shape, lattice="D3Q27", seed=7, T0=1400.0, dx=1e-3, mech=None,
                  amp_T=2e-2, amp_u=3.0, amp_Y=2e-3):
    """A periodic box with seeded temperature, velocity and composition
    perturbations, so that gradients, diffusion velocities and the energy
    flux corrections are all exercised."""
    mech = mech or h2_air_synthetic()
    nx, ny, nz = shape
    rng = philox(seed)
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


def wall_ramp(x, nx, T_cold=300.0, T_hot=1500.0, frac=0.25):
    """Wall temperature: linear T_cold -> T_hot over the first `frac` of the
    length, then T_hot."""
    L = frac * nx
    return np.where(x < L, T_cold + (T_hot - T_cold) * x / L, T_hot)


def channel_2d(seed=0, nx=2000, ny=40, phi=0.5, T_in=300.0, dx=25e-6, steps=50000,
               mech=None, T_wall_hot=1500.0):
    """2-D microchannel: D2Q9 nx x ny, Tamm-Mott-Smith walls beyond y = 0 and
    y = ny-1 carrying the wall_ramp temperature (300 K to T_wall_hot), parabolic inlet
    u = u_max 4 s (1 - s) (s = (y + 1/2)/ny, u_max drawn from the seed in
    [0.2, 3] m/s) of fresh mixture at x = 0, pressure outlet at x = nx-1.
    Initial state: T = wall temperature of the column, fresh mixture, the
    inlet velocity profile everywhere."""
    mech = mech or h2_air_synthetic()
    u_max = float(philox(seed).uniform(0.2, 3.0))
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, phi))
    w = _uniform_fields(mech, (nx, ny, 1), T_in, P_STANDARD, Y)
    x = np.arange(nx, dtype=float)
    s = (np.arange(ny) + 0.5) / ny
    prof = u_max * 4.0 * s * (1.0 - s)
    Tw = wall_ramp(x, nx, T_hot=T_wall_hot)
    w["T"] = np.broadcast_to(Tw[None, None, :], (1, ny, nx)).copy()
    w["u"][0] = np.broadcast_to(prof[None, :, None], (1, ny, nx))
    w.update(lattice="D2Q9", shape=(nx, ny, 1), dx=dx, T_max=3000.0, substeps=2,
             faces=("inlet", "outlet", "tms", "tms", "periodic", "periodic"),
             wall_T=w["T"].copy(),
             inlet=dict(u=w["u"].copy(), T=T_in, Y=Y, P=P_STANDARD),
             outlet=dict(P=P_STANDARD), steps=steps, seed=seed,
             name=f"channel {nx}x{ny} D2Q9 phi={phi} u_max={u_max:.3f}")
    return w


def pipe_wall_geometry(ny, nz, radius):
    """The circular wall (y - c)^2 + (z - c)^2 = radius^2, c = (n-1)/2, as
    grid data: the solid mask of the cross-section, and for every node its
    normal distance to the wall (radius - r) and inward unit normal
    (0, -(y - c)/r, -(z - c)/r).  Returns (solid [nz, ny], dist [nz, ny],
    normal [3, nz, ny])."""
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    zz, yy = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    r = np.sqrt((yy - cy) ** 2 + (zz - cz) ** 2)
    rs = np.where(r > 0, r, 1.0)
    normal = np.stack([np.zeros_like(r), -(yy - cy) / rs, -(zz - cz) / rs])
    return r >= radius, radius - r, normal


def microtube(seed=0, nx=600, ny=40, nz=40, radius=19.0, phi=0.5, T_in=300.0,
              u_in=1.0, dx=25e-6, steps=20000, mech=None, offgrid=False):
    """3-D microtube: D3Q27 nx x ny x nz, fluid where
    (y - c)^2 + (z - c)^2 < radius^2 (c = (ny-1)/2), staircase solid elsewhere
    with Tamm-Mott-Smith walls at the wall_ramp temperature; inlet of fresh
    mixture at u_in at x = 0, pressure outlet at x = nx-1; initial velocity
    u_in (1 + 0.01 N(0,1)) seeded, T = wall temperature of the column.
    offgrid: also give the wall's normal distance and inward normal per node
    (wall_dist, wall_normal), for targets interpolated off the grid."""
    mech = mech or h2_air_synthetic()
    rng = philox(seed)
    Y = mole_to_mass_fractions(mech, air_mole_fractions(mech, phi))
    w = _uniform_fields(mech, (nx, ny, nz), T_in, P_STANDARD, Y)
    x = np.arange(nx, dtype=float)
    cy, cz = (ny - 1) / 2.0, (nz - 1) / 2.0
    zz, yy = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
    fluid2 = (yy - cy) ** 2 + (zz - cz) ** 2 < radius ** 2
    solid = np.broadcast_to(~fluid2[:, :, None], (nz, ny, nx)).copy()
    Tw = wall_ramp(x, nx)
    w["T"] = np.broadcast_to(Tw[None, None, :], (nz, ny, nx)).copy()
    w["u"][0] = u_in * (1.0 + 0.01 * rng.standard_normal((nz, ny, nx)))
    w.update(lattice="D3Q27", shape=(nx, ny, nz), dx=dx, T_max=3000.0, substeps=2,
             faces=("inlet", "outlet", "periodic", "periodic", "periodic", "periodic"),
             solid=solid, solid_kind="tms", wall_T=w["T"].copy(),
             inlet=dict(u=np.array([u_in, 0.0, 0.0]), T=T_in, Y=Y, P=P_STANDARD),
             outlet=dict(P=P_STANDARD), steps=steps, seed=seed,
             name=f"microtube {nx}x{ny}x{nz} D3Q27 r={radius} phi={phi}")
    if offgrid:
        _, dist, normal = pipe_wall_geometry(ny, nz, radius)
        w["wall_dist"] = np.broadcast_to(dist[:, :, None], (nz, ny, nx)).copy()
        w["wall_normal"] = np.broadcast_to(normal[:, :, :, None], (3, nz, ny, nx)).copy()
    return w


def serving_mix(seed=0, n_requests=64, mean_interarrival=0.05, steps=(1000, 10000),
                max_nodes=256 * 32 * 32, mech=None):
    """Seeded request stream for the serving loop: Poisson arrivals (mean
    `mean_interarrival` s), each request a reactor, a flame or a channel solve
    with its type, grid, equivalence ratio in [0.4, 0.7], inlet speed in
    [0.2, 3] m/s and step count drawn from the seed.  Grids range from 16^3
    to max_nodes nodes.  Returns [(arrival_s, workload), ...] sorted by
    arrival; workload["steps"] is the request's step count."""
    mech = mech or h2_air_synthetic()
    rng = philox(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(mean_interarrival))
        kind = ("reactor", "flame", "channel")[int(rng.integers(0, 3))]
        phi = float(rng.uniform(0.4, 0.7))
        u_in = float(rng.uniform(0.2, 3.0))
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        if kind == "reactor":
            nn = int(rng.integers(16, 33))
            # dx = 12.5 um (the flame's spacing) keeps the explicit reaction
            # sub-steps stable through ignition over the full 1k-10k steps:
            # at 1 mm they diverge at ignition, at 50 um within 10k steps
            w = reactor(seed=seed * 1000 + k, n=nn, phi=phi, dx=12.5e-6, mech=mech)
        elif kind == "flame":
            nx = int(rng.choice([256, 512, 1024]))
            ny = int(rng.choice([4, 8, 16, 32]))
            while nx * ny * ny > max_nodes:
                ny //= 2
            w = flame_1d(seed=seed * 1000 + k, nx=nx, ny=ny, nz=ny, phi=phi,
                         x_ign=nx // 4, mech=mech)
            w["inlet"]["u"] = np.array([u_in, 0.0, 0.0])
            w["u"][0] = u_in
        else:
            nx = int(rng.choice([250, 500, 1000, 2000]))
            ny = int(rng.choice([20, 40]))
            # 12.5 um as for the reactors (the channel's own 25 um loses the
            # explicit sub-steps near the hot walls within 10k steps)
            # walls ramping to 1000 K, below the chain-branching crossover of
            # H2/air at 1 atm: with 1500 K walls the preheated mixture
            # autoignites within ~5k steps and a reaction zone that reaches
            # the outlet corner makes the LODI outlet fail (both precisions)
            w = channel_2d(seed=seed * 1000 + k, nx=nx, ny=ny, phi=phi, dx=12.5e-6, mech=mech,
                           T_wall_hot=1000.0)
            s = (np.arange(ny) + 0.5) / ny
            prof = u_in * 4.0 * s * (1.0 - s)
            w["u"][0] = np.broadcast_to(prof[None, :, None], w["u"][0].shape)
            w["inlet"]["u"] = w["u"].copy()
        w["steps"] = nsteps
        w["kind"] = kind
        out.append((t, w))
    return out
