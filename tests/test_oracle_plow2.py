"""Pins for the oracle's quadratic second level (p_low = 2; Section 3: the coarse level is
"a linear or quadratic discretization", Section 3.1.2 transfers between the spaces).

Independent references: scipy B-splines with numpy Gauss quadrature for the mixed mass
and for the 2h -> h embedding (coefficients of each coarse function in the fine basis by
least squares on many points), the closed-form quadratic subdivision weights, the
Galerkin identities of nested spaces, and the dense two-level error propagation
(I - R^T A_c^{-1} R A) S_E built with numpy.  The paper prints no p_low = 2 numbers for
the square, so these are the pins; parity of the method itself is pinned by the
mathematics only.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from test_oracle_transfers import _mixed_mass_scipy


def _basis_values(xi, k, nfun, xs):
    out = np.empty((nfun, xs.size))
    for i in range(nfun):
        c = np.zeros(nfun)
        c[i] = 1.0
        out[i] = BSpline(xi, c, k, extrapolate=False)(xs)
    return np.nan_to_num(out)[1:-1]


@pytest.mark.parametrize("p", [2, 3, 4, 5, 8])
def test_mixed_mass_to_quadratic_against_scipy(oracle_mod, p):
    m = 9
    Mx = oracle_mod.mixed_mass_1d(p, 2, m)
    ref = _mixed_mass_scipy(p, 2, m, oracle_mod.knots(p, m), oracle_mod.knots(2, m))
    assert Mx.shape == (m, m + p - 2)
    assert np.allclose(Mx, ref, atol=1e-15)


@pytest.mark.parametrize("mc", [4, 7, 10])
def test_quadratic_embedding(oracle_mod, mc):
    """Coarse quadratic B-splines written in the fine basis: least squares on 40 points per
    fine element reproduces S (nested spaces: the fit is exact), interior columns carry
    the subdivision weights 1/4, 3/4, 3/4, 1/4, and S^T M_f S = M_c, S^T K_f S = K_c."""
    S = oracle_mod.embed_spline(2, mc)
    mf = 2 * mc
    assert S.shape == (mf, mc)
    xs = np.linspace(0.0, 1.0, 40 * mf + 1)[:-1] + 0.5 / (40 * mf)
    Bf = _basis_values(oracle_mod.knots(2, mf), 2, mf + 2, xs)
    Bc = _basis_values(oracle_mod.knots(2, mc), 2, mc + 2, xs)
    ref, *_ = np.linalg.lstsq(Bf.T, Bc.T, rcond=None)
    assert np.abs(S - ref).max() <= 1e-12
    for I in range(1, mc - 1):   # interior coarse functions: support away from the boundary
        col = S[:, I]
        nz = np.nonzero(np.abs(col) > 1e-14)[0]
        assert np.allclose(col[nz], [0.25, 0.75, 0.75, 0.25], atol=1e-14)
    Kf, Mf = oracle_mod.assemble_1d(2, mf)
    Kc, Mc = oracle_mod.assemble_1d(2, mc)
    assert np.abs(S.T @ Mf @ S - Mc).max() <= 1e-15
    assert np.abs(S.T @ Kf @ S - Kc).max() <= 1e-12 * np.abs(Kc).max()


@pytest.mark.parametrize("mc", [4, 9])
def test_general_embedding_reduces_to_nodal_for_linears(oracle_mod, mc):
    assert np.abs(oracle_mod.embed_spline(1, mc) - oracle_mod.embed_p1(mc)).max() <= 1e-15


@pytest.mark.parametrize("p", [3, 5])
@pytest.mark.parametrize("aggressive", [False, True])
def test_quadratic_restriction(oracle_mod, p, aggressive):
    """R = [S^T] D^{-1} M_p^2: interior rows of D^{-1} M_p^2 sum to 1 (the lumped projection
    reproduces constants away from the boundary); the aggressive form is S^T times it;
    the p_low = 1 path of the general routine equals or_restriction_1d."""
    m = 16
    R0 = oracle_mod.restriction_plow(p, 2, m, aggressive=False)
    Mx = _mixed_mass_scipy(p, 2, m, oracle_mod.knots(p, m), oracle_mod.knots(2, m))
    _, M2 = oracle_mod.assemble_1d(2, m)
    assert np.allclose(R0, Mx / M2.sum(axis=1)[:, None], atol=1e-14)
    rows = R0.sum(axis=1)
    assert np.allclose(rows[p + 1:-(p + 1)], 1.0, atol=1e-13)
    R = oracle_mod.restriction_plow(p, 2, m, aggressive=aggressive)
    if aggressive:
        assert np.allclose(R, oracle_mod.embed_spline(2, m // 2).T @ R0, atol=1e-14)
    else:
        assert np.array_equal(R, R0)
    assert np.array_equal(oracle_mod.restriction_plow(p, 1, m, aggressive), oracle_mod.restriction_1d(p, m, aggressive))


@pytest.mark.parametrize("p,m,aggressive", [(3, 8, True), (4, 10, True), (3, 8, False)])
def test_quadratic_two_level_cycle_matches_dense_formula(oracle_mod, p, m, aggressive):
    """One cycle with the quadratic second level: e_new = (I - R^T A_c^{-1} R A) S_E e,
    A_c the Galerkin degree-2 matrix of the second-level mesh (built here from
    or_assemble_1d(2, .) and numpy Kronecker products)."""
    from test_oracle_cycle import _block, _dense_A
    P = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.EXACT,
                           aggressive=aggressive, plow=2)
    K, M = oracle_mod.assemble_1d(p, m)
    A = _dense_A(K, M, 2)
    N, n = A.shape[0], m + p - 2
    r = (P.s - 1) // 2
    _, order, _ = oracle_mod.schedule(2, n, P.s, p, oracle_mod.LATTICE)
    SE = np.eye(N)
    for c in order:
        B = _block(2, n, c, r)
        V = np.zeros((len(B), N))
        V[np.arange(len(B)), B] = 1.0
        SE = (np.eye(N) - V.T @ np.linalg.solve(V @ A @ V.T, V @ A)) @ SE
    R1 = oracle_mod.restriction_plow(p, 2, m, aggressive=aggressive)
    R = np.kron(R1, R1)
    mc = m // 2 if aggressive else m
    Kc, Mc = oracle_mod.assemble_1d(2, mc)
    Ac = _dense_A(Kc, Mc, 2)
    T = (np.eye(N) - R.T @ np.linalg.solve(Ac, R @ A)) @ SE
    rng = np.random.default_rng(9)
    b, u = rng.standard_normal(N), rng.standard_normal(N)
    ustar = np.linalg.solve(A, b)
    ref = ustar + T @ (u - ustar)
    got = P.cycle(u, b)
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("p", [3, 4, 5])
def test_quadratic_second_level_converges(oracle_mod, p):
    """Measured two-level factor with the quadratic 2h second level (exact solve) on 48^2
    elements: a contraction, no worse than the linear second level's by more than 0.05."""
    m = 48
    rates = {}
    for plow in (1, 2):
        P = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.EXACT, plow=plow)
        rng = np.random.default_rng(p)
        u = rng.uniform(-1, 1, P.N)
        b = np.zeros(P.N)
        r0 = np.linalg.norm(P.residual(u, b))
        for _ in range(12):
            u = P.cycle(u, b)
        rates[plow] = (np.linalg.norm(P.residual(u, b)) / r0) ** (1 / 12)
    assert rates[2] < 0.6
    assert rates[2] <= rates[1] + 0.05, rates
