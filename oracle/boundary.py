"""Boundary conditions of Sec. 4, applied between streaming and collision.

Test infrastructure: plain FP64 numpy, vectorised over interface nodes.

Nomenclature (Sec. 4.1): boundaries lie outside the node layers; a node is an
interface node when some link i has its source x - c_i outside the domain
(beyond a non-periodic face) or on a solid node; those links form the
incoming set D(x).  Each interface node gets one procedure, chosen by the
kinds of the boundaries its incoming links come from, with walls before the
inlet before the outlet:

* bounce-back, Eq. bb: f_i(x) = f_{-i}^post(x) for i in D, all lattices;
* Tamm-Mott-Smith wall, Sec. 4.2.2, Eqs. BBrho-fatms (targets at the node
  itself: u^tgt = u_a^tgt = 0, T^tgt = wall temperature of the node);
* flux inlet, Sec. 4.3, Eqs. in_f-fa_inlet; with spec["inlet"]["simplified"]
  true, the simplified inlet of the same section: stop after the local state
  of step 2 and give every population the local equilibrium (Eqs.
  in_loc_f, in_loc_g, in_loc_fa), so u and T keep their local values;
* outlet, Sec. 4.4, Eqs. convectiveBC-fa_outlet, with the LODI data below.

LODI outlet (Poinsot & Lele 1992; the paper gives no formulas, so this is a
reading): with outward normal n, normal velocity u_n, sound speed
c = sqrt(gamma theta) (gamma = C_p/C_v of the mixture) and one-sided
differences d_n q = q(x) - q(x - n) of the previous step's fields,
  L1 = K (p - p_out),  K = sigma (1 - Ma^2) c / L_n        (incoming wave)
  L2 = u_n (c^2 d_n rho - d_n p)                           (entropy wave)
  L5 = (u_n + c)(d_n p + rho c d_n u_n)                    (outgoing wave)
  Lt = u_n d_n u_t for each tangential component t
and one forward-Euler step (dt = 1) from the previous values at x:
  rho^out = rho - (L2 + (L5 + L1)/2) / c^2,   p^out = p - (L5 + L1)/2,
  u_n^out = u_n - (L5 - L1)/(2 rho c),        u_t^out = u_t - Lt,
  T^out = p^out / (rho^out R(Y^out)).
Mass fractions, Eq. convectiveBC with a backward difference along n:
  Y^out = Y - u_n d_n Y.
"Previous step's fields" are the fields of the stored post-collision state
at time t - dt (what the moments call reports), at x and x - n; before the
first step these are the initial fields.

Gradient ghost values for nodes outside the domain (reading): wall or solid
-> Phi = 0 (the wall is at rest) and Y = Y(x); inlet -> Phi of the inlet
state and Y = Y(x); outlet -> the value at x.
"""
import numpy as np

from . import thermo
from .lattice import normalised_equilibrium, energy_equilibrium
from .lbm import species_velocity_undefined

KINDS = {"periodic": 0, "bounce_back": 1, "tms": 2, "inlet": 3, "outlet": 4}
PRECEDENCE = {1: 3, 2: 3, 3: 2, 4: 1}        # walls > inlet > outlet


class Boundaries:
    """Boundary reconstruction of Sec. 4 for one OracleLBM: face kinds, solid
    nodes, interface-node classification and the procedures of Eq. bb and
    Secs. 4.2.2 (TMS wall), 4.3 (inlet) and 4.4 (LODI outlet)."""

    def __init__(self, lbm, spec):
        self.lbm = lbm
        vs = lbm.vs
        D = vs.dim
        nz, ny, nx = lbm.shape
        ext = (nx, ny, nz)
        faces = [KINDS[f] if isinstance(f, str) else int(f) for f in spec.get("faces", ("periodic",) * 6)]
        self.faces = faces
        self.solid = np.zeros(lbm.shape, dtype=bool) if spec.get("solid") is None \
            else np.asarray(spec["solid"], dtype=bool).reshape(lbm.shape)
        self.solid_kind = KINDS[spec.get("solid_kind", "tms")]
        wall_T = spec.get("wall_T")
        self.wall_T = None if wall_T is None else np.broadcast_to(
            np.asarray(wall_T, dtype=float), lbm.shape).copy()
        inlet = spec.get("inlet")
        outlet = spec.get("outlet", {})
        mech = lbm.mech
        self.outlet_P = float(outlet.get("P", 101325.0))
        self.outlet_sigma = float(outlet.get("sigma", 0.25))
        # LODI length L of K = sigma (1 - Ma^2) c / L: the domain's extent
        # along the outlet normal unless given (a slab of a longer domain
        # keeps the whole domain's length)
        self.outlet_length = outlet.get("length")
        if inlet is not None:
            u_in = np.asarray(inlet["u"], dtype=float)
            if u_in.ndim == 1:                       # uniform, else one vector per node
                u_in = np.broadcast_to(u_in[:, None, None, None], (3,) + lbm.shape)
            self.u_in = u_in.reshape((3,) + lbm.shape)[:D] / lbm.units.c
            self.T_in = float(inlet["T"])
            self.Y_in = np.asarray(inlet["Y"], dtype=float)
            self.inlet_simplified = bool(inlet.get("simplified", False))
            self.rho_in = float(thermo.density_from_pressure(
                mech, float(inlet.get("P", 101325.0)), self.T_in, self.Y_in[:, None])[0])
        # incoming set and the kind of each incoming link
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        coord = (x, y, z)
        self.incoming = np.zeros((vs.Q,) + lbm.shape, dtype=bool)
        link_kind = np.zeros((vs.Q,) + lbm.shape, dtype=int)
        self.out_axis = np.full(lbm.shape, -1)
        self.out_sign = np.zeros(lbm.shape, dtype=int)
        for i, ci in enumerate(vs.c):
            kind = np.zeros(lbm.shape, dtype=int)
            src = []
            for a in range(3):
                if a >= D:
                    src.append(coord[a])
                    continue
                s = coord[a] - ci[a]
                lo, hi = s < 0, s >= ext[a]
                for mask, face in ((lo, 2 * a), (hi, 2 * a + 1)):
                    fk = faces[face]
                    if fk != 0:
                        upd = mask & (PRECEDENCE.get(fk, 0) > np.vectorize(
                            lambda k: PRECEDENCE.get(k, 0))(kind))
                        kind = np.where(upd, fk, kind)
                        if fk == 4:
                            self.out_axis = np.where(mask, a, self.out_axis)
                            self.out_sign = np.where(mask, 1 if face % 2 else -1, self.out_sign)
                src.append(np.mod(s, ext[a]))
            inside = kind == 0
            src_solid = self.solid[src[2], src[1], src[0]]
            kind = np.where(inside & src_solid, self.solid_kind, kind)
            self.incoming[i] = kind != 0
            link_kind[i] = kind
        prec = np.vectorize(lambda k: PRECEDENCE.get(k, 0))(link_kind)
        best = np.argmax(prec, axis=0)
        self.node_kind = np.take_along_axis(link_kind, best[None], axis=0)[0]
        self.node_kind = np.where(self.solid, 0, self.node_kind)
        self.incoming &= ~self.solid[None]
        if np.any((self.node_kind == 2) & (self.wall_T is None)):
            raise ValueError("TMS walls need wall_T")
        self.ext = ext
        self._offgrid_targets(spec)

    def _offgrid_targets(self, spec):
        """Off-grid TMS targets (Sec. 4.2.2, last paragraph; reading R20).
        With spec["wall_dist"] (normal distance delta >= 0 from each node to
        the wall, lattice units) and spec["wall_normal"] ([3, ...] inward
        unit normal n), a TMS node x interpolates its targets linearly along
        the normal between the wall (at -delta) and the fluid node
        x_f = x + c_k (at h = c_k . n), c_k the lattice vector most aligned
        with n:  phi^tgt = (h phi^wall + delta phi(x_f)) / (h + delta), for
        u, u_a (wall values 0) and T.  phi(x_f) are the fields of the stored
        post-collision state of x_f.  Nodes whose x_f is solid or beyond a
        non-periodic face keep the wall values (reading R12)."""
        self.og_nodes = None
        wd, wn = spec.get("wall_dist"), spec.get("wall_normal")
        if wd is None or wn is None:
            return
        lbm = self.lbm
        vs = lbm.vs
        D = vs.dim
        nz, ny, nx = lbm.shape
        ext = (nx, ny, nz)
        wd = np.broadcast_to(np.asarray(wd, dtype=float), lbm.shape).ravel()
        wn = np.asarray(wn, dtype=float).reshape(3, -1)[:D]
        c = vs.c.astype(float)
        nonzero = np.array([i for i in range(vs.Q) if np.any(vs.c[i])])
        cn = c[nonzero] / np.linalg.norm(c[nonzero], axis=1)[:, None]
        nodes, nbr, h, delta = [], [], [], []
        for node in np.nonzero((self.node_kind == 2).ravel())[0]:
            n_hat = wn[:, node]
            k = nonzero[int(np.argmax(cn @ n_hat))]
            xyz = [node % nx, (node // nx) % ny, node // (nx * ny)]
            ok = True
            for a in range(D):
                s_a = xyz[a] + int(vs.c[k][a])
                if s_a < 0 or s_a >= ext[a]:
                    if self.faces[2 * a + (1 if s_a >= ext[a] else 0)] != 0:
                        ok = False
                    s_a %= ext[a]
                xyz[a] = s_a
            f = xyz[0] + nx * (xyz[1] + ny * xyz[2])
            if not ok or self.solid.ravel()[f]:
                continue
            nodes.append(node)
            nbr.append(f)
            h.append(float(c[k] @ n_hat))
            delta.append(float(wd[node]))
        self.og_nodes = np.array(nodes, dtype=int)
        self.og_nbr = np.array(nbr, dtype=int)
        self.og_h = np.array(h)
        self.og_delta = np.array(delta)

    # ------------------------------------------------------------------ #
    def _equilibria(self, rho, Y, u, T, u_species=None):
        """Equilibrium populations [L, Q, n] of the state (rho, Y, u, T) at n
        nodes (Eqs. faEqGeneral, fEqGeneral, gEqGeneral); species a < M use
        u_species[a] when given, else u."""
        lbm, mech = self.lbm, self.lbm.mech
        M = lbm.M
        c2 = lbm.units.c ** 2
        theta_a = thermo.species_gas_constant(mech)[:, None] * T[None] / c2
        theta = thermo.mixture_gas_constant(mech, Y) * T / c2
        U = thermo.mixture_U(mech, Y, T) / c2
        out = np.empty((lbm.L, lbm.vs.Q, rho.size))
        for a in range(M - 1):
            ua = u if u_species is None else u_species[a]
            out[a] = rho * Y[a] * normalised_equilibrium(lbm.vs, ua, theta_a[a])
        out[M - 1] = rho * normalised_equilibrium(lbm.vs, u, theta)
        out[M] = energy_equilibrium(lbm.vs, rho, u, theta, U)
        return out

    def _local_state(self, p, T_guess):
        """rho, u, Y, u_species, T of populations p [L, Q, n] (Eqs. locRho-locT)."""
        lbm = self.lbm
        M = lbm.M
        c = lbm.vs.c.astype(float)
        rho = p[M - 1].sum(axis=0)
        j = c.T @ p[M - 1]
        rs = np.empty((M, rho.size))
        js = np.empty((M, lbm.vs.dim, rho.size))
        for a in range(M - 1):
            rs[a] = p[a].sum(axis=0)
            js[a] = c.T @ p[a]
        rs[M - 1] = rho - rs[: M - 1].sum(axis=0)
        js[M - 1] = j - js[: M - 1].sum(axis=0)
        u = j / rho
        Y = rs / rho
        bad = np.array([species_velocity_undefined(rs[a], js[a]) for a in range(M)])
        us = np.where(bad[:, None], u[None], js / np.where(bad, 1.0, rs)[:, None])
        E = p[M].sum(axis=0) / rho
        U = (E - 0.5 * np.sum(u ** 2, axis=0)) * lbm.units.c ** 2
        T = thermo.temperature_from_energy(lbm.mech, Y, U, T_guess, lbm.newton_rtol,
                                           lbm.newton_max_iter)
        return rho, u, Y, us, T

    def apply(self, post, pops):
        """Replace the incoming populations of every interface node (Sec. 4:
        Eq. bb, Secs. 4.2.2, 4.3, 4.4; walls before inlet before outlet)."""
        lbm = self.lbm
        out = pops.copy()
        flat = out.reshape(lbm.L, lbm.vs.Q, -1)
        post_flat = post.reshape(lbm.L, lbm.vs.Q, -1)
        inc_flat = self.incoming.reshape(lbm.vs.Q, -1)
        kind = self.node_kind.ravel()
        Tguess = lbm.T.ravel()
        opp = lbm.vs.opposite
        for k in (1, 2, 3, 4):
            idx = np.nonzero(kind == k)[0]
            if idx.size == 0:
                continue
            p = flat[:, :, idx]
            D = inc_flat[:, idx][None]                         # [1, Q, n]
            if k == 1:                                         # bounce-back, Eq. bb
                bb = post_flat[:, opp][:, :, idx]
                flat[:, :, idx] = np.where(D, bb, p)
            elif k == 2:
                flat[:, :, idx] = self._tms(p, post_flat[:, opp][:, :, idx], D, idx, Tguess[idx],
                                            post_flat)
            elif k == 3:
                flat[:, :, idx] = self._inlet(p, D, idx, Tguess[idx])
            else:
                flat[:, :, idx] = self._outlet(p, D, idx, Tguess[idx], post)
        return out

    def _tms(self, p, bb, D, idx, Tg, post_flat=None):
        """Sec. 4.2.2, steps 1-4."""
        lbm = self.lbm
        M, dim = lbm.M, lbm.vs.dim
        n = idx.size
        # step 1: bounce-back density and mass fractions (Eqs. BBrho, BBY)
        pb = np.where(D, bb, p)
        rho_bb = pb[M - 1].sum(axis=0)
        Y_bb = np.empty((M, n))
        for a in range(M - 1):
            Y_bb[a] = pb[a].sum(axis=0) / rho_bb
        Y_bb[M - 1] = 1.0 - Y_bb[: M - 1].sum(axis=0)
        # step 2: target equilibria at (rho_bb, Y_bb, u_wall = 0, T_wall), or
        # at the off-grid targets interpolated towards the fluid
        u_t = np.zeros((dim, n))
        T_t = self.wall_T.ravel()[idx].copy()
        us_t = None
        if self.og_nodes is not None and self.og_nodes.size:
            pos = np.searchsorted(self.og_nodes, idx)
            pos = np.minimum(pos, self.og_nodes.size - 1)
            has = self.og_nodes[pos] == idx
            if np.any(has):
                sel = np.nonzero(has)[0]
                j = pos[sel]
                pf = post_flat[:, :, self.og_nbr[j]]
                _, u_f, _, us_f, T_f = self._local_state(pf, Tg[sel])
                h, dl = self.og_h[j], self.og_delta[j]
                w = dl / (h + dl)
                us_t = np.zeros((M, dim, n))
                u_t[:, sel] = w * u_f
                us_t[:, :, sel] = w * us_f
                T_t[sel] = (h * T_t[sel] + dl * T_f) / (h + dl)
        tgt = self._equilibria(rho_bb, Y_bb, u_t, T_t, u_species=us_t)
        # step 3: local state with the incoming populations at the target
        pl = np.where(D, tgt, p)
        rho_l, u_l, Y_l, us_l, T_l = self._local_state(pl, Tg)
        loc = self._equilibria(rho_l, Y_l, u_l, T_l, u_species=us_l)
        # step 4, Eqs. ftms, gtms, fatms
        return np.where(D, 2.0 * tgt - loc, tgt + p - loc)

    def _inlet(self, p, D, idx, Tg):
        """Sec. 4.3, steps 1-4."""
        lbm = self.lbm
        n = p.shape[-1]
        rho_in = np.full(n, self.rho_in)
        Y_in = np.repeat(self.Y_in[:, None], n, axis=1)
        u_in = self.u_in.reshape(self.u_in.shape[0], -1)[:, idx]
        T_in = np.full(n, self.T_in)
        fin = self._equilibria(rho_in, Y_in, u_in, T_in)              # Eqs. in_f-in_fa
        pl = np.where(D, fin, p)
        rho_l, u_l, Y_l, _, T_l = self._local_state(pl, Tg)           # Eqs. inletlocRho-T
        loc = self._equilibria(rho_l, Y_l, u_l, T_l)                  # Eqs. in_loc_*
        if self.inlet_simplified:
            return loc                                                # simplified inlet
        tgt = self._equilibria(rho_l, Y_l, u_in, T_in)                # Eqs. in_tgt_*
        return np.where(D, tgt + fin - loc, tgt + p - loc)            # Eqs. f_inlet-fa_inlet

    def stored_fields(self, post, nodes):
        """rho, u, T, Y of the stored post-collision state `post` at flat node
        indices (the fields at time t - dt that Eq. convectiveBC and the LODI
        data take); Newton starts from the T field."""
        lbm = self.lbm
        p = post.reshape(lbm.L, lbm.vs.Q, -1)[:, :, nodes]
        rho, u, Y, _, T = self._local_state(p, lbm.T.ravel()[nodes])
        return rho, u, T, Y

    def lodi_state(self, idx, post):
        """LODI outlet data (Sec. 4.4, Eq. convectiveBC; reading R13) (rho, u, T,
        Y) at outlet nodes idx (flat), from the
        stored state of the previous step at x and x - n."""
        lbm = self.lbm
        mech = lbm.mech
        dim = lbm.vs.dim
        nz, ny, nx = lbm.shape
        ax = self.out_axis.ravel()[idx]
        sg = self.out_sign.ravel()[idx]
        stride = np.array([1, nx, nx * ny])
        up = idx - sg * stride[ax]                                    # upstream node x - n
        rho0, u0, T0, Y0 = self.stored_fields(post, idx)
        rho1, u1, T1, Y1 = self.stored_fields(post, up)
        c2 = lbm.units.c ** 2
        R0 = thermo.mixture_gas_constant(mech, Y0)
        R1 = thermo.mixture_gas_constant(mech, Y1)
        p0 = rho0 * R0 * T0 / c2
        p1 = rho1 * R1 * T1 / c2
        cols = np.arange(idx.size)
        un0 = sg * u0[ax, cols]
        un1 = sg * u1[ax, cols]
        Cv = thermo.mixture_Cv(mech, Y0, T0)
        gamma = (Cv + R0) / Cv
        cs = np.sqrt(gamma * R0 * T0 / c2)
        Ma = un0 / cs
        Ln = np.array([nx, ny, nz])[ax] if self.outlet_length is None else \
            np.full(idx.size, float(self.outlet_length))
        K = self.outlet_sigma * (1.0 - Ma ** 2) * cs / Ln
        P_t = self.outlet_P / c2
        dn_rho = rho0 - rho1
        dn_p = p0 - p1
        dn_un = un0 - un1
        L1 = K * (p0 - P_t)
        L2 = un0 * (cs ** 2 * dn_rho - dn_p)
        L5 = (un0 + cs) * (dn_p + rho0 * cs * dn_un)
        rho_o = rho0 - (L2 + 0.5 * (L5 + L1)) / cs ** 2
        p_o = p0 - 0.5 * (L5 + L1)
        un_o = un0 - (L5 - L1) / (2.0 * rho0 * cs)
        u_o = np.empty((dim, idx.size))
        for a in range(dim):
            ut = u0[a]
            u_o[a] = ut - un0 * (ut - u1[a])                           # tangential: u_n d_n u_t
        u_o[ax, cols] = sg * un_o
        Y_o = Y0 - un0[None] * (Y0 - Y1)                               # Eq. convectiveBC
        T_o = p_o * c2 / (rho_o * thermo.mixture_gas_constant(mech, Y_o))
        return rho_o, u_o, T_o, Y_o

    def _outlet(self, p, D, idx, Tg, post):
        """Sec. 4.4, steps 1-3."""
        rho_o, u_o, T_o, Y_o = self.lodi_state(idx, post)
        fout = self._equilibria(rho_o, Y_o, u_o, T_o)                 # Eqs. out_f-out_fa
        pl = np.where(D, fout, p)
        rho_l, u_l, Y_l, _, T_l = self._local_state(pl, Tg)           # Eqs. outletloc*
        loc = self._equilibria(rho_l, Y_l, u_l, T_l)
        return np.where(D, 2.0 * fout - loc, fout + p - loc)          # Eqs. f_outlet-fa_outlet

    # ------------------------------------------------------------------ #
    def gradient(self, lbm, phi, kind):
        """Isotropic gradient (Sec. 3.4, readings R7, R8) with ghost values
        outside the fluid (see the module docstring).  phi: [K, z, y, x]; kind: "Phi" or "Y"."""
        vs = lbm.vs
        D = vs.dim
        nz, ny, nx = lbm.shape
        ext = (nx, ny, nz)
        z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        coord = (x, y, z)
        if kind == "Phi":
            theta_in = thermo.mixture_gas_constant(lbm.mech, self.Y_in[:, None])[0] * self.T_in \
                / lbm.units.c ** 2 if hasattr(self, "u_in") else 0.0
            phi_in = (self.rho_in * self.u_in * (1.0 - 3.0 * theta_in)
                      - self.rho_in * self.u_in ** 3) if hasattr(self, "u_in") else None
            # phi_in: [D, z, y, x], the inlet state at each node's own inlet velocity
        grads = np.zeros((D,) + phi.shape)
        for i, ci in enumerate(vs.c):
            if not np.any(ci):
                continue
            kindmap = np.zeros(lbm.shape, dtype=int)
            src = []
            for a in range(3):
                if a >= D:
                    src.append(coord[a])
                    continue
                s = coord[a] + ci[a]
                for mask, face in ((s < 0, 2 * a), (s >= ext[a], 2 * a + 1)):
                    fk = self.faces[face]
                    if fk != 0:
                        kindmap = np.where(mask & (kindmap == 0), fk, kindmap)
                src.append(np.mod(s, ext[a]))
            nb = phi[:, src[2], src[1], src[0]]
            nb_solid = self.solid[src[2], src[1], src[0]]
            kindmap = np.where((kindmap == 0) & nb_solid, self.solid_kind, kindmap)
            wall = (kindmap == 1) | (kindmap == 2)
            inl = kindmap == 3
            outl = kindmap == 4
            if kind == "Phi":
                ghost = np.where(wall[None], 0.0, nb)
                if phi_in is not None:
                    ghost = np.where(inl[None], phi_in, ghost)
                ghost = np.where(outl[None], phi, ghost)
            else:
                ghost = np.where((wall | inl | outl)[None], phi, nb)
            for a in range(D):
                if ci[a] != 0:
                    grads[a] = grads[a] + 3.0 * vs.w[i] * ci[a] * ghost
        return grads
