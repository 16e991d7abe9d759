"""Flame diagnostics of a state: the quantities the paper follows in its
microchannel and microtube runs (Sec. 5.3: the integrated heat release rate,
normalised by that of the unburnt state; the heat release rate field; the
position where the flame begins; the maximum temperature and velocity).

Test infrastructure: plain FP64 numpy.

* Heat release rate per unit volume, q = -sum_a H_a(T) rho_dot_a (W/m^3),
  with H_a the mass-specific enthalpy including the enthalpy of formation
  (Sec. 3.1) and rho_dot_a the mass production rates of the mechanism
  (Sec. 2.4).  Endothermic nodes give q < 0.
* Integrated heat release rate: the sum of q over the nodes times the cell
  volume dx^3 (W) in 3-D, or the cell area dx^2 (W per metre of depth) in 2-D.
* Flame position: the coordinate x = i dx (m) along the first axis of the node
  with the largest q; among equal maxima the one with the smallest node index
  (x fastest).
* T_max (K) and u_max = the largest |u| (m/s).
"""
import numpy as np

from . import chemistry, thermo


def heat_release_rate(mech, T, rho_species):
    """q (W/m^3) at each node (Sec. 5.3 follows it; q = -sum_a H_a rho_dot_a
    with H_a of Sec. 3.1); T: [...], rho_species: [M, ...]."""
    wdot = chemistry.production_rates(mech, T, rho_species)
    return -np.sum(thermo.H_species(mech, T) * wdot, axis=0)


def diagnostics(mech, rho, u, T, Y, dx, dim, nx, fluid=None):
    """rho [N], u [D or 3, N] (m/s), T [N], Y [M, N] of the N = nx*ny*nz nodes
    (x fastest); fluid: optional [N] bool mask (solid nodes excluded).
    Returns dict(hrr_integral, hrr_max, flame_x, T_max, u_max)."""
    rho = np.asarray(rho, float).reshape(-1)
    T = np.asarray(T, float).reshape(-1)
    Y = np.asarray(Y, float).reshape(mech.n_species, -1)
    u = np.asarray(u, float)
    u = u.reshape(u.shape[0], -1)          # [D or 3, N]
    keep = np.ones(rho.size, bool) if fluid is None else np.asarray(fluid, bool).reshape(-1)
    q = heat_release_rate(mech, T, rho * Y)
    qk = np.where(keep, q, -np.inf)
    n_max = int(np.argmax(qk))          # first index of the maximum
    speed = np.sqrt(np.sum(u[:dim] ** 2, axis=0))
    return dict(
        hrr_integral=float(np.sum(q[keep]) * dx ** dim),
        hrr_max=float(q[n_max]),
        flame_x=float((n_max % nx) * dx),
        T_max=float(np.max(T[keep])),
        u_max=float(np.max(speed[keep])),
    )
