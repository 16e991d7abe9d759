"""Pins of the oracle's lattice layer against facts fixed by the paper and by
the mathematics (not by retyping the oracle's formulas).

* Product form, Sec. 2.2: its moments are the parameters it is built from,
  sum Psi = 1, sum Psi c_a = xi_a, sum Psi c_a^2 = P_aa, sum Psi c_a c_b =
  xi_a xi_b (a != b).
* Energy equilibrium, Sec. 3.4, Eq. geq_i: the closed form equals a symbolic
  application of the operators O_a = theta d/du_a + u_a to E, and its
  moments are Eqs. geq1mom and geq2mom.
* Isotropic gradient: exact on linear fields.
"""
import itertools

import numpy as np
import pytest

from oracle.lattice import (VelocitySet, product_form, normalised_equilibrium,
                            energy_equilibrium)


@pytest.mark.parametrize("dim", [2, 3])
def test_velocity_set_structure(dim):
    vs = VelocitySet(dim)
    assert vs.Q == 3 ** dim
    # every combination of {-1,0,1}^D appears once, rest velocity in the middle
    assert len({tuple(c) for c in vs.c}) == vs.Q
    assert np.all(vs.c[vs.Q // 2] == 0)
    assert np.all(vs.c[vs.opposite] == -vs.c)
    assert np.all(vs.opposite == vs.Q - 1 - np.arange(vs.Q))
    # x is the fastest-running component of the index
    assert tuple(vs.c[1][:2]) == (0, -1) and tuple(vs.c[0][:2]) == (-1, -1)
    # weights: sum 1, second moment 1/3 (standard isotropic lattice)
    assert np.isclose(vs.w.sum(), 1.0, atol=1e-15)
    for a in range(dim):
        for b in range(dim):
            m2 = np.sum(vs.w * vs.c[:, a] * vs.c[:, b])
            assert np.isclose(m2, (1.0 / 3.0) if a == b else 0.0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_product_form_moments(dim):
    vs = VelocitySet(dim)
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.uniform(-0.2, 0.2, dim)
        P = rng.uniform(0.05, 0.6, dim) + xi ** 2
        psi = product_form(vs, xi, P)
        c = vs.c.astype(float)
        assert abs(psi.sum() - 1.0) < 1e-15
        for a in range(dim):
            assert abs(np.sum(psi * c[:, a]) - xi[a]) < 1e-15
            assert abs(np.sum(psi * c[:, a] ** 2) - P[a]) < 1e-15
            for b in range(dim):
                if b != a:
                    assert abs(np.sum(psi * c[:, a] * c[:, b]) - xi[a] * xi[b]) < 1e-15


def test_species_equilibrium_moments():
    """Eq. 27eq: sum f^eq = rho_a, sum f^eq c = rho_a u, sum f^eq c c =
    rho_a (R_a T I + u u)."""
    vs = VelocitySet(3)
    u = np.array([0.03, -0.02, 0.01])
    theta = 0.2
    psi = normalised_equilibrium(vs, u, theta)
    c = vs.c.astype(float)
    P2 = np.einsum("i,ia,ib->ab", psi, c, c)
    assert np.allclose(P2, theta * np.eye(3) + np.outer(u, u), atol=1e-16)


def _symbolic_geq(dim):
    sp = pytest.importorskip("sympy")
    u = sp.symbols("u0:%d" % dim)
    th, U = sp.symbols("theta U")
    E = U + sum(x ** 2 for x in u) / 2

    def O(A, a):
        return th * sp.diff(A, u[a]) + u[a] * A

    def psi_op(cval, A, a):
        OA = O(A, a)
        O2A = O(OA, a)
        if cval == 0:
            return A - O2A
        if cval == 1:
            return (OA + O2A) / 2
        return (-OA + O2A) / 2

    vs = VelocitySet(dim)
    exprs = []
    for ci in vs.c:
        A = E
        for a in range(dim):
            A = psi_op(int(ci[a]), A, a)
        exprs.append(sp.lambdify((u, th, U), sp.expand(A), "numpy"))
    return vs, exprs


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_equilibrium_matches_operator_definition(dim):
    vs, exprs = _symbolic_geq(dim)
    rng = np.random.default_rng(2)
    for _ in range(5):
        u = rng.uniform(-0.1, 0.1, dim)
        theta = rng.uniform(0.01, 0.4)
        U = rng.uniform(-3.0, 3.0)
        rho = rng.uniform(0.2, 2.0)
        g = energy_equilibrium(vs, rho, u, theta, U)
        ref = np.array([rho * e(tuple(u), theta, U) for e in exprs])
        assert np.allclose(g, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_equilibrium_moments(dim):
    """Eq. geq1mom: q^eq = (H + u^2/2) rho u; Eq. geq2mom:
    R^eq = (H + u^2/2) P^eq + P u u, with H = U + theta, P = rho theta and
    P^eq = rho theta I + rho u u; and sum g^eq = rho E (Eq. g0momTotalEnergy)."""
    vs = VelocitySet(dim)
    c = vs.c.astype(float)
    u = np.array([0.04, -0.03, 0.02])[:dim]
    theta, U, rho = 0.05, -1.7, 0.8
    g = energy_equilibrium(vs, rho, u, theta, U)
    E = U + 0.5 * u @ u
    Htot = U + theta + 0.5 * u @ u
    assert np.isclose(g.sum(), rho * E, rtol=1e-14)
    assert np.allclose(c.T @ g, Htot * rho * u, rtol=1e-13, atol=1e-16)
    Peq = rho * theta * np.eye(dim) + rho * np.outer(u, u)
    Req = Htot * Peq + rho * theta * np.outer(u, u)
    assert np.allclose(np.einsum("i,ia,ib->ab", g, c, c), Req, rtol=1e-13, atol=1e-16)


def test_gradient_exact_on_linear_fields():
    from oracle.lbm import OracleLBM
    from lbm_workloads.mechanism import binary_inert
    o = OracleLBM(binary_inert(), "D3Q27", (8, 7, 6), 1e-3, c_ref=300.0)
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    phi = 0.3 * x - 1.1 * y + 2.5 * z + 4.0
    grad = o.gradient(phi)
    inner = (slice(1, -1),) * 3
    assert np.allclose(grad[0][inner], 0.3, atol=1e-13)
    assert np.allclose(grad[1][inner], -1.1, atol=1e-13)
    assert np.allclose(grad[2][inner], 2.5, atol=1e-13)
    # D2Q9
    o2 = OracleLBM(binary_inert(), "D2Q9", (9, 5, 1), 1e-3, c_ref=300.0)
    y2, x2 = np.meshgrid(np.arange(5), np.arange(9), indexing="ij")
    phi2 = (-0.7 * x2 + 0.25 * y2)[None]
    g2 = o2.gradient(phi2)
    assert np.allclose(g2[0][0, 1:-1, 1:-1], -0.7, atol=1e-13)
    assert np.allclose(g2[1][0, 1:-1, 1:-1], 0.25, atol=1e-13)


def test_opposite_and_index_convention_documented():
    """The population index convention is part of the C-ABI: i = (cz+1)*9 +
    (cy+1)*3 + (cx+1) (D3Q27) and (cy+1)*3 + (cx+1) (D2Q9)."""
    for dim in (2, 3):
        vs = VelocitySet(dim)
        for i, ci in enumerate(vs.c):
            idx = sum((int(ci[a]) + 1) * 3 ** a for a in range(dim))
            assert idx == i
    assert list(itertools.islice(VelocitySet(2).opposite, 3)) == [8, 7, 6]
