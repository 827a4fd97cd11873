"""Pins for the oracle's splines, quadrature and 1D assembly (Section 2.1).

Every check here is independent of the oracle's own formulas: scipy's B-spline
implementation, closed forms of cardinal B-splines in exact rational
arithmetic, basic invariants, and the O(h^{p+1}) convergence of the Galerkin
solution to the manufactured solution of Section 5.1.
"""
import json
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest
from scipy.interpolate import BSpline

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_knot_vector(oracle_mod):
    # Section 2.1: p+1 zeros, interior knots i/m, p+1 ones
    for p, m in [(1, 3), (2, 5), (5, 4)]:
        xi = oracle_mod.knots(p, m)
        assert len(xi) == 2 * p + m + 1
        assert np.all(xi[: p + 1] == 0.0) and np.all(xi[-(p + 1):] == 1.0)
        assert np.allclose(xi[p: p + m + 1], np.arange(m + 1) / m, atol=0, rtol=0)


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("m", [1, 3, 10])
def test_partition_of_unity_and_nonnegativity(oracle_mod, p, m):
    for x in np.linspace(0.0, 1.0, 41):
        N, dN = oracle_mod.basis_eval(p, m, x)
        assert abs(N.sum() - 1.0) < 1e-14
        assert N.min() >= 0.0
        assert abs(dN.sum()) < 1e-10 * (m + p)  # derivative of a constant


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8])
def test_basis_matches_scipy(oracle_mod, p):
    m = 7
    xi = oracle_mod.knots(p, m)
    xs = np.linspace(0.0, 1.0 - 1e-12, 57)
    for i in range(m + p):
        c = np.zeros(m + p)
        c[i] = 1.0
        spl = BSpline(xi, c, p, extrapolate=False)
        ref = spl(xs)
        dref = spl.derivative()(xs)
        got = np.array([oracle_mod.basis_eval(p, m, x)[0][i] for x in xs])
        dgot = np.array([oracle_mod.basis_eval(p, m, x)[1][i] for x in xs])
        assert np.allclose(got, ref, atol=1e-13)
        assert np.allclose(dgot, dref, atol=1e-10 * m ** 1)


def test_right_endpoint(oracle_mod):
    # N_{m+p}(1) = 1, all others vanish (last span closed on the right)
    for p in range(1, 6):
        N, _ = oracle_mod.basis_eval(p, 4, 1.0)
        assert N[-1] == 1.0 and np.all(N[:-1] == 0.0)


@pytest.mark.parametrize("npts", range(1, 12))
def test_gauss_exactness(oracle_mod, npts):
    x, w = oracle_mod.gauss(npts)
    for k in range(2 * npts):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-14
    xr, wr = np.polynomial.legendre.leggauss(npts)
    assert np.allclose(np.sort(x), np.sort(xr), atol=1e-14)


@pytest.mark.parametrize("p", range(1, 9))
def test_full_matrices_invariants(oracle_mod, p):
    m = 12
    K, M = oracle_mod.assemble_1d(p, m, full=True)
    assert np.allclose(K, K.T, atol=1e-13) and np.allclose(M, M.T, atol=1e-16)
    # constants lie in the full space: K 1 = 0, 1^T M 1 = |Omega| = 1
    assert np.abs(K.sum(axis=1)).max() < 1e-11 * m
    assert abs(M.sum() - 1.0) < 1e-13
    # band structure: supports overlap only within p
    i, j = np.indices(K.shape)
    assert np.all(K[np.abs(i - j) > p] == 0.0) and np.all(M[np.abs(i - j) > p] == 0.0)
    # restricted space drops the first and last function (eq. splinespace)
    Kr, Mr = oracle_mod.assemble_1d(p, m)
    assert np.array_equal(Kr, K[1:-1, 1:-1]) and np.array_equal(Mr, M[1:-1, 1:-1])
    assert np.all(np.linalg.eigvalsh(Kr) > 0)


def _cardinal(n, x, deriv=0):
    """Centred cardinal B-spline of degree n and its derivatives, exact rationals.
    B_n(x) = 1/n! sum_j (-1)^j C(n+1,j) (x + (n+1)/2 - j)_+^n."""
    tot = Fraction(0)
    for j in range(n + 2):
        t = Fraction(x) + Fraction(n + 1, 2) - j
        if t <= 0:
            continue
        pw = n - deriv
        coef = Fraction(factorial(n), factorial(pw)) if deriv else 1
        tot += (-1) ** j * comb(n + 1, j) * coef * t ** pw
    return tot / factorial(n)


@pytest.mark.parametrize("p", range(1, 9))
def test_interior_rows_match_cardinal_closed_form(oracle_mod, p):
    """Interior rows of M and K are Toeplitz: M_k = h B_{2p+1}(k), K_k = -B''_{2p+1}(k)/h."""
    m = 4 * p + 8
    K, M = oracle_mod.assemble_1d(p, m)
    h = 1.0 / m
    i = (m + p - 2) // 2
    for k in range(-p, p + 1):
        mk = float(_cardinal(2 * p + 1, k)) * h
        kk = -float(_cardinal(2 * p + 1, k, deriv=2)) / h
        assert abs(M[i, i + k] - mk) < 1e-15
        assert abs(K[i, i + k] - kk) < 1e-12 * m


def test_stencil_golden_fractions(oracle_mod):
    with open(os.path.join(GOLDEN, "stencils_1d.json")) as fh:
        gold = json.load(fh)
    for p_str, ent in gold["stencils"].items():
        p = int(p_str)
        m = 4 * p + 8
        K, M = oracle_mod.assemble_1d(p, m)
        i = (m + p - 2) // 2
        kh = [float(Fraction(v)) for v in ent["K_times_h"]]
        mh = [float(Fraction(v)) for v in ent["M_over_h"]]
        assert np.allclose(K[i, i - p: i + p + 1] / m, kh, atol=1e-14, rtol=0)
        assert np.allclose(M[i, i - p: i + p + 1] * m, mh, atol=1e-15, rtol=0)


def _l2_error(oracle_mod, p, m, u):
    """|| u_h - sin(pi x) sin(pi y) ||_L2 with 6 Gauss points per element per axis."""
    gx, gw = np.polynomial.legendre.leggauss(p + 4)
    h = 1.0 / m
    xs = (np.arange(m)[:, None] * h + 0.5 * h * (gx[None, :] + 1.0)).ravel()
    ws = np.tile(0.5 * h * gw, m)
    B = np.array([oracle_mod.basis_eval(p, m, x)[0][1:-1] for x in xs])  # restricted basis
    n = m + p - 2
    U = B @ u.reshape(n, n).T @ B.T  # U[a,b] = u_h(x_a, y_b); u[j, i] is x-index i
    ex = np.outer(np.sin(np.pi * xs), np.sin(np.pi * xs))
    return np.sqrt(np.einsum("a,b,ab->", ws, ws, (U - ex) ** 2))


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_l2_convergence_rate(oracle_mod, p):
    """Section 5.1 problem: -Lap u = 2 pi^2 sin sin; Galerkin error O(h^{p+1})."""
    errs = []
    ms = [4, 8, 16]
    for m in ms:
        K, M = oracle_mod.assemble_1d(p, m)
        A = np.kron(K, M) + np.kron(M, K)
        g = oracle_mod.load_1d(p, m, kind=0)
        b = 2.0 * np.pi ** 2 * np.kron(g, g)
        u = np.linalg.solve(A, b)
        errs.append(_l2_error(oracle_mod, p, m, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.25, (errs, rates)


def test_load_vector_against_scipy_quadrature(oracle_mod):
    from scipy.integrate import quad
    p, m = 3, 6
    xi = oracle_mod.knots(p, m)
    g = oracle_mod.load_1d(p, m, kind=1, par=(0.37, 0.05), nq=12)
    for i in range(m + p - 2):
        c = np.zeros(m + p)
        c[i + 1] = 1.0
        spl = BSpline(xi, c, p)
        ref = quad(lambda x: np.exp(-0.5 * ((x - 0.37) / 0.05) ** 2) * spl(x), 0, 1,
                   points=list(np.arange(1, m) / m), limit=200, epsabs=1e-15)[0]
        assert abs(g[i] - ref) < 1e-11
