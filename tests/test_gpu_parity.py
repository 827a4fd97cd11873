"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: FP64 per-iterate agreement to 1e-12 relative (2-norm), and
element-wise agreement to 1e-12 of the vector's max for single steps.  Sizes
span several tiles with ragged tails; the full 1024^2 workload is checked on
properties the oracle can evaluate at that size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3)}


def _pair(oracle_mod, p, m, coarse="vcycle", sched="lattice"):
    q, g = COLOURING[p]
    cg = iga2l.COARSE_VCYCLE if coarse == "vcycle" else iga2l.COARSE_EXACT
    co = oracle_mod.VCYCLE if coarse == "vcycle" else oracle_mod.EXACT
    sg = iga2l.SCHED_TILE if sched == "tile" else iga2l.SCHED_LATTICE
    so = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    S = iga2l.Solver(p, m, period=q, stride=g, coarse=cg, schedule=sg)
    O = oracle_mod.Problem(2, p, m, sched=so, tile=S.tile or 32, coarse=co, period=q, stride=g,
                           groups=S.tile_groups)
    assert S.N == O.N and S.Nc == O.Nc
    assert (S.period, S.stride) == (q, g)
    return S, O


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _close(got, ref, tol=TOL):
    scale = max(np.abs(ref).max(), 1e-300)
    err = np.abs(got - ref).max() / scale
    assert err <= tol, f"max rel diff {err:.3e} > {tol:.0e}"


def _inputs(N, seed):
    return synth.coefficients(N, seed), synth.initial_guess(N, seed + 1)


CASES = [(2, 24), (2, 50), (3, 26), (3, 64), (4, 30), (4, 66), (5, 28), (5, 70)]


@pytest.mark.parametrize("p,m", CASES)
def test_residual_and_apply(oracle_mod, p, m):
    S, O = _pair(oracle_mod, p, m)
    b, u = _inputs(S.N, 10 * p + m)
    d = torch.empty(S.N, dtype=torch.float64, device="cuda")
    nrm = S.residual(_dev(u), _dev(b), d, want_norm=True)
    dref = O.residual(u, b)
    _close(_host(d), dref)
    assert abs(nrm - np.linalg.norm(dref)) <= TOL * np.linalg.norm(dref)
    y = torch.empty_like(d)
    S.apply_A(_dev(u), y)
    _close(_host(y), O.apply_A(u))


@pytest.mark.parametrize("p,m", CASES + [(2, 100), (5, 132)])
@pytest.mark.parametrize("reverse", [False, True])
@pytest.mark.parametrize("sched", ["lattice", "tile"])
def test_schwarz_sweep(oracle_mod, p, m, reverse, sched):
    S, O = _pair(oracle_mod, p, m, sched=sched)
    b, u = _inputs(S.N, 7 * p + m)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b), reverse=reverse)
    kind = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    _, order, _ = oracle_mod.schedule(2, S.n, O.s, p, kind, S.tile or 32, *COLOURING[p], S.tile_groups)
    if reverse:
        order = order[::-1].copy()
    K, M = oracle_mod.assemble_1d(p, m)
    ref = oracle_mod.schwarz_sweep(2, K, M, p, O.s, order, b, u)
    _close(_host(ud), ref)


@pytest.mark.parametrize("p,m,groups", [(2, 100, 2), (2, 100, 7), (3, 108, 3), (4, 92, 2), (5, 132, 4),
                                        (5, 70, 100)])
@pytest.mark.parametrize("reverse", [False, True])
def test_grouped_tile_sweep(oracle_mod, p, m, groups, reverse):
    """TILE with the colours split into groups (each group runs the four tile phases):
    FP64 sweep against the oracle's grouped order (or_schedule_grouped), per iterate."""
    q, g = COLOURING[p]
    S = iga2l.Solver(p, m, period=q, stride=g, schedule=iga2l.SCHED_TILE, tile_groups=groups)
    assert S.tile_groups == min(groups, q * q)
    O = oracle_mod.Problem(2, p, m, sched=oracle_mod.TILE, tile=S.tile, period=q, stride=g, groups=S.tile_groups)
    b, u = _inputs(S.N, 11 * p + m + groups)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b), reverse=reverse)
    _, order, _ = oracle_mod.schedule(2, S.n, O.s, p, oracle_mod.TILE, S.tile, q, g, S.tile_groups)
    if reverse:
        order = order[::-1].copy()
    K, M = oracle_mod.assemble_1d(p, m)
    _close(_host(ud), oracle_mod.schwarz_sweep(2, K, M, p, O.s, order, b, u))
    # a whole grouped cycle against the oracle's
    ud = _dev(u)
    S.cycle(ud, _dev(b))
    _close(_host(ud), O.cycle(u, b))


@pytest.mark.parametrize("p,m", CASES)
def test_transfers(oracle_mod, p, m):
    S, O = _pair(oracle_mod, p, m)
    d, u = _inputs(S.N, 3 * p + m)
    ec = synth.uniform_pm1(99 + m, S.Nc)
    dc = torch.empty(S.Nc, dtype=torch.float64, device="cuda")
    S.restrict(_dev(d), dc)
    _close(_host(dc), O.restrict(d))
    ud = _dev(u)
    S.prolong_add(_dev(ec), ud)
    _close(_host(ud), O.prolong_add(ec, u))


@pytest.mark.parametrize("p,m,coarse", [(2, 32, "exact"), (2, 64, "vcycle"), (3, 132, "vcycle"),
                                        (4, 40, "exact"), (5, 264, "vcycle")])
def test_coarse_solve(oracle_mod, p, m, coarse):
    S, O = _pair(oracle_mod, p, m, coarse)
    dc = synth.uniform_pm1(5 + m, S.Nc)
    ec = torch.empty(S.Nc, dtype=torch.float64, device="cuda")
    S.coarse_solve(_dev(dc), ec)
    _close(_host(ec), O.coarse_solve(dc))


@pytest.mark.parametrize("p,m", [(2, 50), (3, 64), (4, 66), (5, 70)])
@pytest.mark.parametrize("sched", ["lattice", "tile"])
def test_cycles_per_iterate(oracle_mod, p, m, sched):
    """Per-iterate parity over 5 cycles of Algorithm 1 (V(1,1) second level)."""
    S, O = _pair(oracle_mod, p, m, sched=sched)
    f, u0 = _inputs(S.N, 100 + p)
    K, M = oracle_mod.assemble_1d(p, m)
    b = (M @ f.reshape(S.n, S.n) @ M.T).ravel()
    ud, bd = _dev(u0), _dev(b)
    uo = u0.copy()
    for k in range(5):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        got = _host(ud)
        rel = np.linalg.norm(got - uo) / np.linalg.norm(uo)
        assert rel <= TOL, f"cycle {k + 1}: {rel:.3e}"


def test_config0_manufactured_solution_ten_cycles(oracle_mod):
    """2D p=2 on 32x32 elements, f = 2 pi^2 sin sin, exact second level, 10 cycles."""
    S, O = _pair(oracle_mod, 2, 32, "exact")
    g = oracle_mod.load_1d(2, 32, kind=0)
    b = 2.0 * np.pi ** 2 * np.kron(g, g)
    u0 = synth.initial_guess(S.N, synth.BASE_SEED)
    ud, bd = _dev(u0), _dev(b)
    uo = u0.copy()
    for k in range(10):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        rel = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
        assert rel <= TOL, f"cycle {k + 1}: {rel:.3e}"


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_solve_matches_oracle_counts(oracle_mod, p):
    m = 128
    S, O = _pair(oracle_mod, p, m)
    f, u0 = _inputs(S.N, 200 + p)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    K, M = oracle_mod.assemble_1d(p, m)
    b = (M @ f.reshape(S.n, S.n) @ M.T).ravel()
    _close(_host(bd), b)
    ud = _dev(u0)
    cyc, rel, hist, ok = S.solve_load(bd, ud, tol=1e-8, max_cycles=40)
    uo, cyc_o, rel_o, hist_o, ok_o = O.solve(b, u0, tol=1e-8, maxc=40)
    assert ok and ok_o and cyc == cyc_o
    assert np.allclose(hist, hist_o, rtol=1e-6, atol=0)
    assert np.linalg.norm(_host(ud) - uo) <= TOL * np.linalg.norm(uo)


@pytest.mark.parametrize("p", [2, 5])
def test_solve_takes_coefficients(oracle_mod, p):
    """iga2l_solve(f): the right-hand side is the source's B-spline coefficient vector f,
    b = (f, phi_i) = (M x M) f is formed by the library (Section 2); cycle counts and the
    converged solution match the oracle solving with its own (M x M) f, and the iterates
    equal iga2l_solve_load given the library's b bit for bit."""
    m = 96
    S, O = _pair(oracle_mod, p, m)
    f, u0 = _inputs(S.N, 900 + p)
    K, M = oracle_mod.assemble_1d(p, m)
    b = (M @ f.reshape(S.n, S.n) @ M.T).ravel()
    ud = _dev(u0)
    cyc, rel, hist, ok = S.solve(_dev(f), ud, tol=1e-8, max_cycles=40)
    uo, cyc_o, rel_o, hist_o, ok_o = O.solve(b, u0, tol=1e-8, maxc=40)
    assert ok and ok_o and cyc == cyc_o
    assert np.allclose(hist, hist_o, rtol=1e-6, atol=0)
    assert np.linalg.norm(_host(ud) - uo) <= TOL * np.linalg.norm(uo)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    ul = _dev(u0)
    cl, rl, hl, okl = S.solve_load(bd, ul, tol=1e-8, max_cycles=40)
    assert okl and cl == cyc and np.array_equal(hl, hist) and torch.equal(ul, ud)
    # a handle built with rhs = IGA2L_RHS_IS_LOAD reads b from iga2l_solve
    Sl = iga2l.Solver(p, m, period=S.period, stride=S.stride, rhs=iga2l.RHS_IS_LOAD)
    ub = _dev(u0)
    cb, rb, hb, okb = Sl.solve(bd, ub, tol=1e-8, max_cycles=40)
    assert okb and cb == cyc and np.array_equal(hb, hist) and torch.equal(ub, ud)


def test_adjoint_cycle_identity(oracle_mod):
    """<C x, y> = <x, C^T y> for the GPU cycle and its transpose."""
    S, _ = _pair(oracle_mod, 3, 40)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(S.N), rng.standard_normal(S.N)
    cx = _dev(np.zeros(S.N))
    S.cycle(cx, _dev(x))
    cty = _dev(np.zeros(S.N))
    S.cycle(cty, _dev(y), adjoint=True)
    lhs, rhs = np.dot(_host(cx), y), np.dot(x, _host(cty))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(_host(cx)) * np.linalg.norm(y)


def test_adjoint_solve_matches_oracle(oracle_mod):
    S, O = _pair(oracle_mod, 2, 64)
    gvec, l0 = _inputs(S.N, 77)
    ld = _dev(l0)
    cyc, rel, ok = S.adjoint_solve(_dev(gvec), ld, tol=1e-10, max_cycles=40)
    lo, cyc_o, rel_o, _, ok_o = O.solve(gvec, l0, tol=1e-10, maxc=40, adjoint=True)
    assert ok and ok_o and cyc == cyc_o
    assert np.linalg.norm(_host(ld) - lo) <= TOL * np.linalg.norm(lo)


@pytest.mark.parametrize("p", [2, 5])
def test_full_size_cycle_and_solve(oracle_mod, p):
    """1024x1024 elements (the benchmark workload): one cycle against the oracle, and
    the converged GPU solution's residual re-evaluated by the oracle."""
    m = 1024
    q, g = COLOURING[p]
    S = iga2l.Solver(p, m, period=q, stride=g)
    O = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE,
                           period=q, stride=g)
    f, u0 = _inputs(S.N, 300 + p)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    b = _host(bd)
    ud = _dev(u0)
    S.cycle(ud, bd)
    if p == 2:   # one oracle cycle at this size takes a few seconds for p=2
        uo = O.cycle(u0, b)
        assert np.linalg.norm(_host(ud) - uo) <= TOL * np.linalg.norm(uo)
    ud = _dev(u0)
    cyc, rel, hist, ok = S.solve_load(bd, ud, tol=1e-8, max_cycles=40)
    assert ok and rel <= 1e-8 and 3 <= cyc <= 20
    r_end = np.linalg.norm(O.residual(_host(ud), b))
    r_0 = np.linalg.norm(O.residual(u0, b))
    assert r_end <= 1.0001e-8 * r_0


def test_invalid_calls_raise_before_launch():
    S = iga2l.Solver(2, 24)
    with pytest.raises(ValueError):
        S.cycle(torch.zeros(5, dtype=torch.float64, device="cuda"),
                torch.zeros(S.N, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        S.cycle(torch.zeros(S.N, dtype=torch.float32, device="cuda"),
                torch.zeros(S.N, dtype=torch.float64, device="cuda"))
    # non-finite data is reported, not silently iterated
    b = torch.zeros(S.N, dtype=torch.float64, device="cuda")
    b[3] = float("nan")
    with pytest.raises(iga2l.IgaError) as ei:
        S.solve_load(b, torch.zeros_like(b))
    assert ei.value.code == iga2l.ERR_NONFINITE
    # zero right-hand side and guess: converged with zero cycles
    cyc, rel, hist, ok = S.solve_load(torch.zeros_like(b), torch.zeros_like(b))
    assert ok and cyc == 0


def test_graph_replay_matches_plain_launches(oracle_mod):
    """Cycles replayed from captured CUDA graphs equal plain launches bit for bit."""
    q, g = COLOURING[3]
    A = iga2l.Solver(3, 66, period=q, stride=g, graphs=1)
    B = iga2l.Solver(3, 66, period=q, stride=g, graphs=0)
    f, u0 = _inputs(A.N, 55)
    b = _dev(f)
    ua, ub = _dev(u0), _dev(u0)
    for _ in range(3):
        A.cycle(ua, b)
        B.cycle(ub, b)
    assert torch.equal(ua, ub)
    ua2, ub2 = _dev(u0), _dev(u0)
    ca, ra, ha, _ = A.solve_load(b, ua2, tol=1e-9)
    cb, rb, hb, _ = B.solve_load(b, ub2, tol=1e-9)
    assert ca == cb and np.array_equal(ha, hb) and torch.equal(ua2, ub2)
    n0 = iga2l.kernel_launches()
    A.cycle(ua, b)
    assert iga2l.kernel_launches() - n0 > 30      # a replayed graph still counts its kernels
