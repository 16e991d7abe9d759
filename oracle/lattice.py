"""Velocity sets, product-form populations and the equilibria of the model.

Test infrastructure: plain FP64 numpy, written for reading, not speed.

* Velocity sets: D3Q27, c_ia in {-1, 0, 1} (Sec. 2.2, Eq. d3q27vel); D2Q9 is
  the same product construction on two axes (the paper's 2-D runs do not
  print their lattice; this is the reading used throughout).
* Population index: i = (cz+1)*9 + (cy+1)*3 + (cx+1) for D3Q27 and
  i = (cy+1)*3 + (cx+1) for D2Q9, so the opposite of i is Q-1-i.
* Product form (Sec. 2.2, Eqs. phi0, phiPlus, phis, prod): per axis
  Psi_0 = 1 - P, Psi_{+1} = (xi + P)/2, Psi_{-1} = (-xi + P)/2, and
  Psi_i = prod_alpha Psi_{c_ia}(xi_alpha, P_alpha_alpha).
"""
import itertools

import numpy as np


class VelocitySet:
    """D3Q27 / D2Q9 velocities and the index map of the module docstring
    (Sec. 2.2, Eq. d3q27vel; reading R1)."""

    def __init__(self, dim: int):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        if dim == 3:
            c = [(cx, cy, cz) for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3)]
        else:
            c = [(cx, cy) for cy, cx in itertools.product((-1, 0, 1), repeat=2)]
        self.c = np.array(c, dtype=np.int64)            # [Q, D]
        self.Q = len(c)
        self.opposite = np.array([self._index(tuple(-v)) for v in self.c])
        # isotropic weights of the standard lattice (products of 2/3, 1/6, 1/6
        # per axis): used only by the gradient stencil (reading R7).
        w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
        self.w = np.array([np.prod([w1[int(a)] for a in v]) for v in self.c])
        self.name = "D3Q27" if dim == 3 else "D2Q9"

    def _index(self, v):
        for i, ci in enumerate(self.c):
            if tuple(ci) == tuple(v):
                return i
        raise KeyError(v)


def psi_axis(c, xi, P):
    """One-axis factor Psi_c(xi, P) for c in {-1, 0, 1} (Eqs. phi0-phis)."""
    if c == 0:
        return 1.0 - P
    if c == 1:
        return 0.5 * (xi + P)
    return 0.5 * (-xi + P)


def product_form(vs: VelocitySet, xi, P):
    """Psi_i for all i (Eq. prod).  xi, P: arrays [D, ...] of the per-axis
    parameters xi_alpha and P_alpha_alpha.  Returns [Q, ...]."""
    out = []
    for ci in vs.c:
        term = 1.0
        for a in range(vs.dim):
            term = term * psi_axis(int(ci[a]), xi[a], P[a])
        out.append(term)
    return np.array(out)


def normalised_equilibrium(vs, u, theta):
    """psi_i(u, theta) = Psi_i(xi = u, P_aa = theta + u_a^2): the species
    equilibrium per unit density (Eq. 27eq with rho_a factored out), formed
    directly so that zero densities need no division (reading R4)."""
    u = np.asarray(u)
    P = np.array([theta + u[a] ** 2 for a in range(vs.dim)])
    return product_form(vs, u, P)


def species_equilibrium(vs, rho_a, u, theta_a):
    """f_ai^eq = rho_a Psi(u, R_a T + u^2)  (Eq. 27eq)."""
    return rho_a * normalised_equilibrium(vs, u, theta_a)


def extended_equilibrium(vs, rho, u, P_ex):
    """f_i^ex = rho Psi(u, P^ex_aa)  (Eq. feqmix)."""
    return rho * product_form(vs, np.asarray(u), np.asarray(P_ex))


def energy_equilibrium(vs, rho, u, theta, U):
    """g_i^eq of Eq. geq_i in closed form.

    E = U + sum_a u_a^2/2 with U independent of u, and O_a acts on u_a only, so
    the operator product form separates per axis.  With
        A_c(a) = Psi_c(u_a, theta + u_a^2)           (operators acting on 1)
        B_c(a) = Psi_c(O_a, O_a^2)[u_a^2/2]
    where O_a[u_a^2/2] = theta u_a + u_a^3/2 and
          O_a^2[u_a^2/2] = theta^2 + 5/2 theta u_a^2 + u_a^4/2,
    g_i^eq = rho [U prod_a A + sum_b B_b prod_{a != b} A_a].
    The tests check this against a symbolic application of the operators.
    """
    u = np.asarray(u)
    A, B = [], []
    for a in range(vs.dim):
        ua = u[a]
        O1 = theta * ua + 0.5 * ua ** 3
        O2 = theta ** 2 + 2.5 * theta * ua ** 2 + 0.5 * ua ** 4
        A.append({0: 1.0 - (theta + ua ** 2), 1: 0.5 * (ua + theta + ua ** 2),
                  -1: 0.5 * (-ua + theta + ua ** 2)})
        B.append({0: 0.5 * ua ** 2 - O2, 1: 0.5 * (O1 + O2), -1: 0.5 * (-O1 + O2)})
    out = []
    for ci in vs.c:
        prodA = 1.0
        for a in range(vs.dim):
            prodA = prodA * A[a][int(ci[a])]
        term = U * prodA
        for b in range(vs.dim):
            t = B[b][int(ci[b])]
            for a in range(vs.dim):
                if a != b:
                    t = t * A[a][int(ci[a])]
            term = term + t
        out.append(rho * term)
    return np.array(out)
