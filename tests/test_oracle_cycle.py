"""Pins for the oracle's two-level cycle (Algorithm 1), the degree-1 V(1,1)
cycle (Section 3.2), the adjoint cycle and the solver's stopping rule.

Independent references: the paper's error-propagation formula
(I - P A_c^{-1} R A) S_p built densely with numpy; symmetry/adjoint identities
that hold for any correct implementation; the dense direct solution; and, as
soft pins, the convergence factors and iteration counts the paper prints
(Tables 1, 3 and 4, tests/golden/paper_tables.json).
"""
import json
import os

import numpy as np
import pytest

from paper_2009_01499_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def _kron_list(mats):
    out = mats[0]
    for m_ in mats[1:]:
        out = np.kron(m_, out)
    return out


def _dense_A(K, M, dim):
    if dim == 2:
        return np.kron(K, M) + np.kron(M, K)
    return np.kron(K, np.kron(M, M)) + np.kron(M, np.kron(K, M)) + np.kron(M, np.kron(M, K))


def _block(dim, n, c, r):
    cz, cy, cx = (c // (n * n), (c // n) % n, c % n) if dim == 3 else (0, c // n, c % n)
    out = []
    for z in (range(cz - r, cz + r + 1) if dim == 3 else [0]):
        for y in range(cy - r, cy + r + 1):
            for x in range(cx - r, cx + r + 1):
                if 0 <= x < n and 0 <= y < n and 0 <= z < (n if dim == 3 else 1):
                    out.append(x + n * (y + n * z))
    return np.array(out)


@pytest.mark.parametrize("dim,p,m,kind", [(2, 2, 8, 1), (2, 3, 8, 2), (2, 5, 6, 1), (2, 6, 8, 1), (2, 7, 8, 1),
                                          (3, 2, 4, 1)])
def test_cycle_matches_dense_error_propagation(oracle_mod, dim, p, m, kind):
    """e_new = (I - R^T A_c^{-1} R A) S_E e with exact coarse solve (Sections 3.1, 3.3, 4.1)."""
    P = oracle_mod.Problem(dim, p, m, sched=kind, tile=7, coarse=oracle_mod.EXACT)
    K, M = oracle_mod.assemble_1d(p, m)
    A = _dense_A(K, M, dim)
    N = A.shape[0]
    n = m + p - 2
    r = (P.s - 1) // 2
    _, order, _ = oracle_mod.schedule(dim, n, P.s, p, kind, 7)
    SE = np.eye(N)
    for c in order:
        B = _block(dim, n, c, r)
        V = np.zeros((len(B), N))
        V[np.arange(len(B)), B] = 1.0
        SE = (np.eye(N) - V.T @ np.linalg.solve(V @ A @ V.T, V @ A)) @ SE
    R1 = oracle_mod.restriction_1d(p, m, aggressive=True)
    R = _kron_list([R1] * dim)
    Kc, Mc = oracle_mod.assemble_1d(1, m // 2)
    Ac = _dense_A(Kc, Mc, dim)
    T = (np.eye(N) - R.T @ np.linalg.solve(Ac, R @ A)) @ SE
    rng = np.random.default_rng(2)
    b = rng.standard_normal(N)
    u = rng.standard_normal(N)
    ustar = np.linalg.solve(A, b)
    got = P.cycle(u, b)
    ref = ustar + T @ (u - ustar)
    assert np.allclose(got, ref, atol=1e-10 * np.abs(ref).max())


@pytest.mark.parametrize("dim,m", [(2, 32), (3, 16)])
def test_vcycle_is_symmetric_and_converges(oracle_mod, dim, m):
    """Red-black GS pre-smoothing with the reversed post-smoother makes V(1,1) symmetric."""
    P = oracle_mod.Problem(dim, 2, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(P.Nc)
    y = rng.standard_normal(P.Nc)
    Bx = P.coarse_solve(x)
    By = P.coarse_solve(y)
    assert abs(np.dot(Bx, y) - np.dot(x, By)) < 1e-12 * np.linalg.norm(Bx) * np.linalg.norm(y)
    # as a stand-alone iteration on the degree-1 problem it converges at a textbook rate
    Kc, Mc = oracle_mod.assemble_1d(1, m // 2)
    Ac = _dense_A(Kc, Mc, dim)
    e = rng.standard_normal(P.Nc)
    rates = []
    for _ in range(8):
        r0 = np.linalg.norm(Ac @ e)
        e = e + P.coarse_solve(-Ac @ e)
        rates.append(np.linalg.norm(Ac @ e) / r0)
    assert max(rates[-3:]) < 0.3


def test_cycle_adjoint_identity(oracle_mod):
    """<C x, y> = <x, C^T y>: the transposed cycle is coarse correction first, then the
    reversed-order Schwarz step."""
    for coarse in (oracle_mod.EXACT, oracle_mod.VCYCLE):
        P = oracle_mod.Problem(2, 3, 24, sched=oracle_mod.TILE, tile=7, coarse=coarse)
        rng = np.random.default_rng(8)
        x = rng.standard_normal(P.N)
        y = rng.standard_normal(P.N)
        z = np.zeros(P.N)
        Cx = P.cycle(z, x)
        Cty = P.cycle(z, y, adjoint=True)
        assert abs(np.dot(Cx, y) - np.dot(x, Cty)) < 1e-12 * np.linalg.norm(Cx) * np.linalg.norm(y)
        assert abs(np.dot(P.cycle(z, x), y) - np.dot(x, P.cycle(z, y))) > 1e-6  # C is not symmetric


def test_config0_exact_second_level(oracle_mod):
    """2D, p=2, 32x32 elements, f = 2 pi^2 sin sin (Section 5.1), exact second level, 10 cycles."""
    P = oracle_mod.Problem(2, 2, 32, sched=oracle_mod.LATTICE, coarse=oracle_mod.EXACT)
    g = oracle_mod.load_1d(2, 32, kind=0)
    b = 2.0 * np.pi ** 2 * np.kron(g, g)
    u0 = synth.initial_guess(P.N, synth.BASE_SEED)
    u, cyc, rel, hist, ok = P.solve(b, u0, tol=1e-30, maxc=10)
    assert cyc == 10
    above_floor = hist[hist > 1e-14]
    assert len(above_floor) >= 5 and np.all(np.diff(above_floor) < 0)
    K, M = oracle_mod.assemble_1d(2, 32)
    ustar = np.linalg.solve(_dense_A(K, M, 2), b)
    assert np.linalg.norm(u - ustar) <= 1e-8 * np.linalg.norm(ustar)
    # Table 3 factor for p=2 (0.1723) bounds the observed contraction
    assert hist[-1] < 0.1723 ** 10


def test_solver_stopping_rule(oracle_mod):
    P = oracle_mod.Problem(2, 2, 16, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    b = synth.coefficients(P.N, 3)
    u0 = synth.initial_guess(P.N, 4)
    u, cyc, rel, hist, ok = P.solve(b, u0, tol=1e-8, maxc=50)
    assert ok and rel <= 1e-8 and hist[-2] > 1e-8 and len(hist) == cyc
    r = P.residual(u, b)
    r0 = P.residual(u0, b)
    assert abs(np.linalg.norm(r) / np.linalg.norm(r0) - rel) < 1e-12
    # zero right-hand side and zero guess: converged before any cycle
    _, cyc0, _, _, ok0 = P.solve(np.zeros(P.N), np.zeros(P.N))
    assert ok0 and cyc0 == 0


def _window_rate(oracle_mod, p, m, aggressive, k0=5, k1=20):
    """Geometric mean of the residual reduction per cycle over cycles k0+1..k1, zero
    right-hand side, random initial guess (the paper's rho_h experiment, Section 4.3).
    The cycle operator is not normal, so single ratios oscillate; the windowed mean is
    the statistic used here (the paper does not state its own)."""
    P = oracle_mod.Problem(2, p, m, sched=oracle_mod.LEX, tile=0, coarse=oracle_mod.EXACT,
                           aggressive=aggressive)
    u = synth.initial_guess(P.N, 99)
    b = np.zeros(P.N)
    logs = []
    for _ in range(k1):
        r0 = np.linalg.norm(P.residual(u, b))
        u = P.cycle(u, b)
        r1 = np.linalg.norm(P.residual(u, b))
        logs.append(np.log(r1 / r0))
        u /= r1
    return float(np.exp(np.mean(logs[k0:])))


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_lexicographic_factors_near_paper_tables(oracle_mod, p):
    """Soft pin: lexicographic Schwarz, exact coarse solve.  Same-mesh second level on
    48x48 elements vs the measured rho_h of Table 1; aggressive (2h) second level on 64x64
    elements vs the LFA rho_2g^ag of Table 3.  The paper's colouring is unknown, so the
    lexicographic order is the comparable one.  Finite grids with Dirichlet boundaries
    converge somewhat faster than the infinite-grid LFA (for p=2 the spectral radius
    grows from 0.069 at m=32 to 0.093 at m=64), hence the one-sided tolerance."""
    col = "9p" if oracle_mod.block_size(p) == 3 else "25p"
    same = _window_rate(oracle_mod, p, 48, False)
    aggr = _window_rate(oracle_mod, p, 64, True)
    t1 = GOLD["table1_rho_h_sameh_exact"][col][str(p)]
    t3 = GOLD["table3_rho_2g_aggressive"][col][str(p)]
    assert t1 - 0.07 <= same <= t1 + 0.02, (same, t1)
    assert t3 - 0.07 <= aggr <= t3 + 0.02, (aggr, t3)


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_iteration_counts_near_table4(oracle_mod, p):
    """Soft pin: cycles to 1e-8 on 128x128 elements, aggressive coarsening + V(1,1),
    coloured Schwarz (this project's colouring) vs Table 4."""
    P = oracle_mod.Problem(2, p, 128, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
    g = oracle_mod.load_1d(p, 128, kind=0)
    b = 2.0 * np.pi ** 2 * np.kron(g, g)
    u0 = synth.initial_guess(P.N, synth.BASE_SEED)
    _, cyc, rel, _, ok = P.solve(b, u0, tol=1e-8, maxc=40)
    paper = GOLD["table4_iterations"]["128"][str(p)]
    assert ok and paper - 2 <= cyc <= paper + 4, (cyc, paper)
