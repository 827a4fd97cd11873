"""Pins for the oracle's transfer operators (Sections 3.1.2, 3.3, 4.1).

Independent references: scipy B-splines with numpy Gauss quadrature for the
mixed mass, the closed-form [1/2, 1, 1/2] degree-1 embedding, the Galerkin
identity of nested degree-1 spaces, and adjointness of restriction and
prolongation.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline


def _mixed_mass_scipy(p, plow, m, xi_p, xi_l):
    gx, gw = np.polynomial.legendre.leggauss(p + plow + 2)
    h = 1.0 / m
    xs = (np.arange(m)[:, None] * h + 0.5 * h * (gx[None, :] + 1.0)).ravel()
    ws = np.tile(0.5 * h * gw, m)

    def basis(xi, k, nfun):
        out = np.empty((nfun, xs.size))
        for i in range(nfun):
            c = np.zeros(nfun)
            c[i] = 1.0
            out[i] = BSpline(xi, c, k)(xs)
        return out[1:-1]

    Bp = basis(xi_p, p, m + p)
    Bl = basis(xi_l, plow, m + plow)
    return (Bl * ws) @ Bp.T


@pytest.mark.parametrize("p", [2, 3, 5, 6, 7, 8])
def test_mixed_mass_against_scipy(oracle_mod, p):
    m = 9
    Mx = oracle_mod.mixed_mass_1d(p, 1, m)
    ref = _mixed_mass_scipy(p, 1, m, oracle_mod.knots(p, m), oracle_mod.knots(1, m))
    assert Mx.shape == (m - 1, m + p - 2)
    assert np.allclose(Mx, ref, atol=1e-15)


def test_mixed_mass_same_degree_is_mass(oracle_mod):
    for p in (1, 2, 4):
        _, M = oracle_mod.assemble_1d(p, 10)
        assert np.allclose(oracle_mod.mixed_mass_1d(p, p, 10), M, atol=1e-16)


def test_embedding_closed_form(oracle_mod):
    mc = 6
    S = oracle_mod.embed_p1(mc)
    ref = np.zeros((2 * mc - 1, mc - 1))
    for I in range(mc - 1):
        ref[2 * I, I] = 0.5
        ref[2 * I + 1, I] = 1.0
        ref[2 * I + 2, I] = 0.5
    assert np.allclose(S, ref, atol=4e-16, rtol=0)  # nodal evaluation, rounding only


@pytest.mark.parametrize("mc", [2, 5, 16])
def test_galerkin_identity_degree1(oracle_mod, mc):
    """Nested degree-1 spaces: S^T K_h S = K_2h and S^T M_h S = M_2h (so S^T A_h S = A_2h)."""
    S = oracle_mod.embed_p1(mc)
    Kh, Mh = oracle_mod.assemble_1d(1, 2 * mc)
    K2, M2 = oracle_mod.assemble_1d(1, mc)
    assert np.allclose(S.T @ Kh @ S, K2, atol=1e-12 * mc)
    assert np.allclose(S.T @ Mh @ S, M2, atol=1e-16)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6, 7, 8])
def test_restriction_composition(oracle_mod, p):
    m = 16
    Mx = _mixed_mass_scipy(p, 1, m, oracle_mod.knots(p, m), oracle_mod.knots(1, m))
    _, M1 = oracle_mod.assemble_1d(1, m)
    D = M1.sum(axis=1)  # row-sum lumping of the restricted degree-1 mass
    same = Mx / D[:, None]
    assert np.allclose(oracle_mod.restriction_1d(p, m, aggressive=False), same, atol=1e-14)
    S = oracle_mod.embed_p1(m // 2)
    assert np.allclose(oracle_mod.restriction_1d(p, m, aggressive=True), S.T @ same, atol=1e-14)
    # rows of D^{-1} M_p^1 away from the boundary sum to one (sum_j N_j = 1 there)
    rows = same.sum(axis=1)
    assert np.allclose(rows[p + 1: -(p + 1)], 1.0, atol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_restrict_prolong_kron_and_adjoint(oracle_mod, dim):
    p, m = 3, 8
    P = oracle_mod.Problem(dim, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.EXACT)
    R = oracle_mod.restriction_1d(p, m, aggressive=True)
    Rk = R
    for _ in range(dim - 1):
        Rk = np.kron(R, Rk)
    rng = np.random.default_rng(5)
    d = rng.standard_normal(P.N)
    e = rng.standard_normal(P.Nc)
    assert np.allclose(P.restrict(d), Rk @ d, atol=1e-13)
    u = rng.standard_normal(P.N)
    assert np.allclose(P.prolong_add(e, u) - u, Rk.T @ e, atol=1e-13)
