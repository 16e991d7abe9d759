"""The reactive-mixture lattice Boltzmann step, written out step by step.

Test infrastructure: plain FP64 numpy; slow and meant to be read beside the
paper.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
use it; the CUDA library never does.

Stored lattices (Sec. 3.7, Eq. strongest): species a = 1..M-1, the momentum
lattice f and the energy lattice g, L = M+1 lattices of Q populations; the
M-th species is slaved, f_Mi = f_i - sum_{a<M} f_ai.  Arrays are
pops[lattice, i, z, y, x] with lattice index 0..M-2 for the species, M-1 for
f and M for g.

Lattice units: dx = dt = 1, velocities in units of the reference speed c
(acoustic scaling, Sec. 3.6), theta_a = R_a T/c^2, theta = R T/c^2, specific
energies divided by c^2, densities kept in kg/m^3.

One step (pull scheme, Sec. 4.1 Eq. advection; then Sec. 2.3 and Sec. 3):
 1. stream all lattices;                      2. boundary reconstruction;
 3. moments;                                  4. temperature (Eq. temperature);
 5. relaxation parameters (Eqs. betaa, taua, mu, lambda);
 6. isotropic gradients of Phi_a = rho u_a (1 - 3 theta) - rho u_a^3 and Y_a;
 7. diffusion velocities V_a (Eq. transform1, Householder QR as in Sec. 2.3);
 8. reaction sub-steps (Eq. R3);
 9. collision of species (Eq. finalNumericalEquationsReactive), momentum
    (Eq. f with the extended equilibrium, Eqs. feqmix and Pex) and energy
    (Eq. g with Eqs. geq_i, gstar, gstareq1mom, qdiff, corrFourier, qex);
10. store.
"""
import numpy as np

from lbm_workloads.mechanism import R_UNIVERSAL
from . import thermo, chemistry, transport
from .lattice import (VelocitySet, normalised_equilibrium, product_form,
                      energy_equilibrium)

RHO_TINY = 1e-300   # below this species density, u_a := u (reading R5)


def species_velocity_undefined(rho_a, j_a):
    """Reading R5 of Eq. momentum1 (u_a = j_a / rho_a): the species velocity
    is replaced by the mixture velocity when rho_a <= 1e-300, or when some
    component satisfies |j_a| >= rho_a.  Non-negative populations always give
    |j_a| <= rho_a, so a species velocity at or beyond the lattice speed only
    arises from cancellation in near-zero densities (after a boundary
    reconstruction); there j_a / rho_a is rounding noise, and the product
    form evaluated at it is unbounded.  rho_a: [...], j_a: [D, ...]."""
    return (rho_a <= RHO_TINY) | np.any(np.abs(j_a) >= rho_a[None], axis=0)


class Units:
    """Acoustic scaling: dt = dx / c (reading R10)."""

    def __init__(self, dx, c):
        self.dx = float(dx)
        self.c = float(c)
        self.dt = self.dx / self.c


def default_reference_speed(mech, T_max):
    """c = sqrt(max_a R_a T_max / 0.9): keeps theta_a + u^2 below 1 for the
    lightest species at T_max, so every product-form factor stays in [0, 1]
    at small u (reading R10)."""
    return float(np.sqrt(np.max(thermo.species_gas_constant(mech)) * T_max / 0.9))


class OracleLBM:
    """The reactive-mixture LBM of Secs. 2-4 on a box of nodes, in plain FP64
    (test infrastructure)."""

    def __init__(self, mech, lattice="D3Q27", shape=(16, 16, 16), dx=1e-3,
                 c_ref=0.0, T_max=3000.0, substeps=2, newton_rtol=1e-13,
                 newton_max_iter=50, boundaries=None):
        self.mech = mech
        self.vs = VelocitySet(3 if lattice == "D3Q27" else 2)
        nx, ny, nz = shape
        if self.vs.dim == 2 and nz != 1:
            raise ValueError("D2Q9 needs nz = 1")
        self.shape = (nz, ny, nx)
        self.M = mech.n_species
        self.L = self.M + 1
        c = c_ref if c_ref > 0 else default_reference_speed(mech, T_max)
        self.units = Units(dx, c)
        self.substeps = int(substeps)
        self.newton_rtol = newton_rtol
        self.newton_max_iter = newton_max_iter
        self.boundaries = boundaries
        if boundaries is not None:
            from .boundary import Boundaries
            self.bc = Boundaries(self, boundaries)
        else:
            self.bc = None
        self.pops = np.zeros((self.L, self.vs.Q) + self.shape)
        self.T = np.zeros(self.shape)
        self.step_count = 0

    # ------------------------------------------------------------------ #
    # helpers
    def _theta_a(self, T):
        Ra = thermo.species_gas_constant(self.mech)
        return Ra.reshape((-1,) + (1,) * np.ndim(T)) * T / self.units.c ** 2

    def _shift(self, field, c):
        """field(x - c) on the periodic grid: np.roll moves a[x] to x + c (the pull
        streaming of Sec. 4.1)."""
        axes = (-1, -2, -3)                          # x, y, z axes of [..., z, y, x]
        out = field
        for a in range(self.vs.dim):
            if c[a] != 0:
                out = np.roll(out, int(c[a]), axis=axes[a])
        return out

    def stream(self, pops):
        """Pull streaming, Eq. advection: f_i(x) = f_i^post(x - c_i)."""
        out = np.empty_like(pops)
        for i, ci in enumerate(self.vs.c):
            out[:, i] = self._shift(pops[:, i], ci)
        return out

    def gradient(self, phi):
        """Isotropic lattice gradient (reading R7):
        d_a phi(x) = 3 sum_i w_i c_ia phi(x + c_i).  phi: [..., z, y, x]."""
        grads = np.zeros((self.vs.dim,) + phi.shape)
        for i, ci in enumerate(self.vs.c):
            nb = self._shift(phi, -ci)
            for a in range(self.vs.dim):
                if ci[a] != 0:
                    grads[a] = grads[a] + 3.0 * self.vs.w[i] * ci[a] * nb
        return grads

    # ------------------------------------------------------------------ #
    def init_fields(self, rho, u, T, Y):
        """Populations at the equilibria of (rho, u, T, Y) (Sec. 4.1,
        Eqs. faEqGeneral, fEqGeneral, gEqGeneral): f_a^eq for a < M, the
        conventional f^eq (Eq. feq) and g^eq.  Inputs in SI units; rho, T
        shaped like the grid [nz, ny, nx] (or flat, x fastest), u [D, ...],
        Y [M, ...]."""
        rho = np.asarray(rho, dtype=float).reshape(self.shape)
        T = np.asarray(T, dtype=float).reshape(self.shape)
        u = np.asarray(u, dtype=float).reshape((-1,) + self.shape)[: self.vs.dim] / self.units.c
        Y = np.asarray(Y, dtype=float).reshape((self.M,) + self.shape)
        theta_a = self._theta_a(T)
        theta = thermo.mixture_gas_constant(self.mech, Y) * T / self.units.c ** 2
        U = thermo.mixture_U(self.mech, Y, T) / self.units.c ** 2
        for a in range(self.M - 1):
            self.pops[a] = rho * Y[a] * normalised_equilibrium(self.vs, u, theta_a[a])
        self.pops[self.M - 1] = rho * normalised_equilibrium(self.vs, u, theta)
        self.pops[self.M] = energy_equilibrium(self.vs, rho, u, theta, U)
        self.T = T.copy()
        if self.bc is not None:
            self.solid_state = self.pops[:, :, self.bc.solid].copy()

    # ------------------------------------------------------------------ #
    def moments_of(self, pops):
        """Moments of a population state (Eqs. density1, momentum1, fdensity,
        f1momMomentum, g0momTotalEnergy, and the slaving Eq. strongest)."""
        M, c = self.M, self.vs.c.astype(float)
        f, g = pops[M - 1], pops[M]
        rho = f.sum(axis=0)
        j = np.einsum("ia,i...->a...", c, f)
        Pten = np.einsum("ia,ib,i...->ab...", c, c, f)
        rho_s = np.zeros((M,) + self.shape)
        j_s = np.zeros((M, self.vs.dim) + self.shape)
        for a in range(M - 1):
            rho_s[a] = pops[a].sum(axis=0)
            j_s[a] = np.einsum("ia,i...->a...", c, pops[a])
        rho_s[M - 1] = rho - rho_s[: M - 1].sum(axis=0)
        j_s[M - 1] = j - j_s[: M - 1].sum(axis=0)
        rhoE = g.sum(axis=0)
        q = np.einsum("ia,i...->a...", c, g)
        return dict(rho=rho, j=j, P=Pten, rho_s=rho_s, j_s=j_s, rhoE=rhoE, q=q)

    def temperature(self, mom, T_guess):
        """Eq. temperature for the moment set `mom` (lattice units in)."""
        rho, j = mom["rho"], mom["j"]
        u = j / rho
        E = mom["rhoE"] / rho
        U_lat = E - 0.5 * np.sum(u ** 2, axis=0)
        Y = mom["rho_s"] / rho
        T = thermo.temperature_from_energy(self.mech, Y, U_lat * self.units.c ** 2,
                                           T_guess, self.newton_rtol, self.newton_max_iter)
        return T, u, Y, U_lat

    # ------------------------------------------------------------------ #
    def step(self, nsteps=1):
        """nsteps time steps of the path (streaming Sec. 4.1, boundaries Sec. 4,
        moments and T Sec. 3.1, sub-steps Sec. 2.4 Eq. R3, collisions Sec. 2.3
        and Secs. 3.2-3.4)."""
        for _ in range(nsteps):
            self._one_step()

    def _one_step(self):
        M, D, vs = self.M, self.vs.dim, self.vs
        c = vs.c.astype(float)
        units = self.units
        # 1. streaming
        post = self.pops
        pops = self.stream(post)
        # 2. boundary reconstruction at interface nodes
        if self.bc is not None:
            pops = self.bc.apply(post, pops)
            if self.bc.solid.any():               # solid nodes stay frozen
                pops[:, :, self.bc.solid] = self.solid_state
        # 3. moments
        mom = self.moments_of(pops)
        rho, rho_s, j_s = mom["rho"], mom["rho_s"], mom["j_s"]
        # 4. temperature (warm start from the previous step's value)
        T, u, Y, U_lat = self.temperature(mom, self.T)
        self.T = T
        u_s = np.empty_like(j_s)
        for a in range(M):
            tiny = species_velocity_undefined(rho_s[a], j_s[a])
            safe = np.where(tiny, 1.0, rho_s[a])
            u_s[a] = np.where(tiny[None], u, j_s[a] / safe[None])
        # 5. relaxation parameters
        rel = transport.relaxation(self.mech, units, rho, Y, T)
        theta, theta_a = rel["theta"], rel["theta_a"]
        omega, omega1 = rel["omega"], rel["omega1"]
        inv_tau_ab, inv_tau_a, beta = rel["inv_tau_ab"], rel["inv_tau_a"], rel["beta"]
        # 6. gradients of Phi_a and Y_a
        Phi = rho[None] * u * (1.0 - 3.0 * theta[None]) - rho[None] * u ** 3
        if self.bc is not None:
            dPhi_all = self.bc.gradient(self, Phi, kind="Phi")
            gradY = self.bc.gradient(self, Y, kind="Y")
        else:
            dPhi_all = self.gradient(Phi)
            gradY = self.gradient(Y)                 # [D, M, ...]
        dPhi = np.array([dPhi_all[a, a] for a in range(D)])   # d_a Phi_a
        # 7. diffusion velocities: A V^alpha = u_a^alpha - u^alpha
        V = self.diffusion_velocities(Y, inv_tau_ab, inv_tau_a, u_s - u[None])
        # 8. reaction sub-steps at frozen U
        drho, _ = chemistry.reactor_substeps(self.mech, rho_s, U_lat * units.c ** 2, T,
                                             units.dt, self.substeps, self.newton_rtol,
                                             self.newton_max_iter)
        # 9. collision
        new = np.empty_like(pops)
        psi_eq = np.array([normalised_equilibrium(vs, u, theta_a[b]) for b in range(M)])
        d = np.empty((M, vs.Q) + self.shape)     # f_b^eq - f_b^*
        for b in range(M):
            xi = u + V[b]
            Pst = np.array([theta_a[b] + xi[a] ** 2 for a in range(D)])
            d[b] = rho_s[b] * (psi_eq[b] - product_form(vs, xi, Pst))
        for a in range(M - 1):
            F = np.zeros((vs.Q,) + self.shape)
            for b in range(M):
                if b != a:
                    F = F + inv_tau_ab[a, b] * d[b]
            F = Y[a] * F
            feq = rho_s[a] * psi_eq[a]
            R = drho[a] * psi_eq[a]
            new[a] = pops[a] + 2.0 * beta[a] * (feq - pops[a]) + (beta[a] - 1.0) * F + R
        # momentum lattice, extended equilibrium
        Pex = np.array([theta + u[a] ** 2 + (2.0 - omega) / (2.0 * rho * omega) * dPhi[a]
                        for a in range(D)])
        fex = rho * product_form(vs, u, Pex)
        f = pops[M - 1]
        new[M - 1] = f + omega * (fex - f)
        # energy lattice
        g = pops[M]
        geq = energy_equilibrium(vs, rho, u, theta, U_lat)
        E = U_lat + 0.5 * np.sum(u ** 2, axis=0)
        q_eq = rho * u * (E + theta)
        Peq = np.zeros((D, D) + self.shape)
        for a in range(D):
            for b in range(D):
                Peq[a, b] = rho * u[a] * u[b] + (rho * theta if a == b else 0.0)
        uP = np.array([sum(u[b] * (mom["P"][b, a] - Peq[b, a]) for b in range(D))
                       for a in range(D)])
        q_ex = np.array([-0.5 * u[a] * dPhi[a] for a in range(D)])
        H_lat = thermo.H_species(self.mech, T) / units.c ** 2          # [M, ...]
        Pres = rho * theta
        diff_flux = np.sum(H_lat[:, None] * Y[:, None] * V, axis=0)     # sum_a H_a Y_a V_a
        corr_flux = np.sum(H_lat[None] * gradY, axis=1)                # sum_a H_a grad Y_a
        W = ((omega - omega1) * (mom["q"] - q_eq - uP + q_ex)
             + omega1 * rho * diff_flux + 0.5 * (2.0 - omega1) * Pres * corr_flux)
        gnew = g + omega * (geq - g)
        for i, ci in enumerate(vs.c):
            if int(np.sum(ci * ci)) == 1:
                gnew[i] = gnew[i] + 0.5 * np.sum(c[i].reshape((-1,) + (1,) * 3) * W, axis=0)
        new[M] = gnew
        # 10. store
        if self.bc is not None:
            if self.bc.solid.any():
                new[:, :, self.bc.solid] = self.solid_state
        self.pops = new
        self.step_count += 1

    def diffusion_velocities(self, Y, inv_tau_ab, inv_tau_a, rhs):
        """Solve Eq. transform1 per node and component by Householder QR.

        A_aa = 1 + 1/(2 tau_a), A_ab = -(1/2) Y_b / tau_ab (b != a);
        rhs: [M, D, ...] = u_a - u.  Returns V [M, D, ...]."""
        M, D = self.M, self.vs.dim
        n = int(np.prod(self.shape))
        A = np.zeros((n, M, M))
        for a in range(M):
            for b in range(M):
                if a == b:
                    A[:, a, a] = (1.0 + 0.5 * inv_tau_a[a]).ravel()
                else:
                    A[:, a, b] = (-0.5 * Y[b] * inv_tau_ab[a, b]).ravel()
        Qm, Rm = np.linalg.qr(A)                        # LAPACK Householder QR
        V = np.zeros((M, D) + self.shape)
        for al in range(D):
            b = np.stack([rhs[a, al].ravel() for a in range(M)], axis=1)   # [n, M]
            y = np.einsum("nba,nb->na", Qm, b)                            # Q^T b
            x = np.zeros_like(y)
            for r in range(M - 1, -1, -1):                                # back substitution
                acc = y[:, r] - np.einsum("nk,nk->n", Rm[:, r, r + 1:], x[:, r + 1:])
                x[:, r] = acc / Rm[:, r, r]
            for a in range(M):
                V[a, al] = x[:, a].reshape(self.shape)
        return V

    # ------------------------------------------------------------------ #
    def moments(self):
        """Fields of the stored post-collision state in SI units (reading
        R14): rho (kg/m^3), u (m/s) [D, ...], T (K), Y [M, ...], E (J/kg)."""
        mom = self.moments_of(self.pops)
        T, u, Y, U_lat = self.temperature(mom, self.T)
        E = mom["rhoE"] / mom["rho"] * self.units.c ** 2
        return dict(rho=mom["rho"], u=u * self.units.c, T=T, Y=Y, E=E)
