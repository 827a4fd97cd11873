"""GPU parity of the 3D path (A = K(x)M(x)M + M(x)K(x)M + M(x)M(x)K, 3x3x3 Schwarz
blocks, 27-point degree-1 hierarchy) against the FP64 oracle, and of the 3D mixed
form against the FP64 GPU form.  The paper is 2D only: these are pinned by the
oracle's own pins (Kronecker apply, product formula, dense cycle formula in 3D)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2)}


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _close(got, ref, tol=TOL):
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err <= tol, f"max rel diff {err:.3e}"


def _pair(oracle_mod, p, m, coarse="vcycle", precision=0):
    q, g = COLOURING[p]
    S = iga2l.Solver(p, m, dim=3, period=q, stride=g, precision=precision,
                     coarse=iga2l.COARSE_VCYCLE if coarse == "vcycle" else iga2l.COARSE_EXACT)
    O = oracle_mod.Problem(3, p, m, sched=oracle_mod.LATTICE, period=q, stride=g,
                           coarse=oracle_mod.VCYCLE if coarse == "vcycle" else oracle_mod.EXACT)
    assert S.N == O.N and S.Nc == O.Nc
    return S, O


@pytest.mark.parametrize("p,m", [(2, 12), (3, 16), (3, 18), (4, 20)])
def test_residual_schwarz_transfers_3d(oracle_mod, p, m):
    S, O = _pair(oracle_mod, p, m)
    b = synth.coefficients(S.N, 3 + p)
    u = synth.initial_guess(S.N, 4 + p)
    d = torch.empty(S.N, dtype=torch.float64, device="cuda")
    nrm = S.residual(_dev(u), _dev(b), d, want_norm=True)
    dref = O.residual(u, b)
    _close(_host(d), dref)
    assert abs(nrm - np.linalg.norm(dref)) <= TOL * np.linalg.norm(dref)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b))
    _close(_host(ud), O.smooth(u, b))
    dc = torch.empty(S.Nc, dtype=torch.float64, device="cuda")
    S.restrict(_dev(dref), dc)
    _close(_host(dc), O.restrict(dref))
    ec = synth.uniform_pm1(9, S.Nc)
    ud = _dev(u)
    S.prolong_add(_dev(ec), ud)
    _close(_host(ud), O.prolong_add(ec, u))
    f = torch.empty_like(d)
    S.rhs_from_coeffs(_dev(b), f)
    K, M = oracle_mod.assemble_1d(p, m)
    n = S.n
    ref = np.einsum("ai,bj,ck,kji->cba", M, M, M, b.reshape(n, n, n)).ravel()
    _close(_host(f), ref)


@pytest.mark.parametrize("m,coarse", [(16, "exact"), (32, "vcycle")])
def test_coarse_solve_3d(oracle_mod, m, coarse):
    S, O = _pair(oracle_mod, 3, m, coarse)
    dc = synth.uniform_pm1(17, S.Nc)
    ec = torch.empty(S.Nc, dtype=torch.float64, device="cuda")
    S.coarse_solve(_dev(dc), ec)
    _close(_host(ec), O.coarse_solve(dc))


def test_cycles_per_iterate_3d(oracle_mod):
    S, O = _pair(oracle_mod, 3, 32)
    b = synth.coefficients(S.N, 21)
    u0 = synth.initial_guess(S.N, 22)
    ud, bd = _dev(u0), _dev(b)
    uo = u0.copy()
    for k in range(3):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        rel = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
        assert rel <= TOL, (k, rel)


def test_mixed_3d_matches_fp64_gpu():
    """3D p = 3 on 64^3 elements: the mixed form takes the FP64 form's cycle count at
    1e-8 and, refined to a 1e-12 residual, is within 1e-8 of its solution."""
    p, m = 3, 64
    q, g = COLOURING[p]
    A = iga2l.Solver(p, m, dim=3, period=q, stride=g)
    B = iga2l.Solver(p, m, dim=3, period=q, stride=g, precision=iga2l.MIXED_FP32)
    f = _dev(synth.coefficients(A.N, 41))
    b = torch.empty_like(f)
    A.rhs_from_coeffs(f, b)
    u0 = _dev(synth.initial_guess(A.N, 42))
    ua, ub = u0.clone(), u0.clone()
    ca, ra, _, oka = A.solve_load(b, ua, tol=1e-8)
    cb, rb, _, okb = B.solve_load(b, ub, tol=1e-8)
    assert oka and okb and abs(ca - cb) <= 1 and 3 <= ca <= 20
    ua, ub = u0.clone(), u0.clone()
    A.solve_load(b, ua, tol=1e-12, max_cycles=60)
    B.solve_load(b, ub, tol=1e-12, max_cycles=60)
    err = float(torch.linalg.norm(ua - ub) / torch.linalg.norm(ua))
    assert err <= 1e-8, err


def _tile_pair(oracle_mod, p, m, precision=0):
    q, g = COLOURING[p]
    S = iga2l.Solver(p, m, dim=3, period=q, stride=g, precision=precision, schedule=iga2l.SCHED_TILE)
    O = oracle_mod.Problem(3, p, m, sched=oracle_mod.TILE, tile=S.tile, period=q, stride=g,
                           coarse=oracle_mod.VCYCLE)
    assert S.tile == q   # the 3D TILE side is the colour period
    return S, O


@pytest.mark.parametrize("p,m", [(2, 12), (3, 16), (3, 20), (4, 20)])
@pytest.mark.parametrize("reverse", [False, True])
def test_schwarz_tile_3d(oracle_mod, p, m, reverse):
    """3D TILE sweep (tile side = colour period, 8 tile phases, ragged last tiles) against
    the oracle's TILE order, forward and reverse."""
    S, O = _tile_pair(oracle_mod, p, m)
    b, u = synth.coefficients(S.N, 50 + p), synth.initial_guess(S.N, 51 + p)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b), reverse=reverse)
    q, g = COLOURING[p]
    _, order, _ = oracle_mod.schedule(3, S.n, O.s, p, oracle_mod.TILE, S.tile, q, g)
    if reverse:
        order = order[::-1].copy()
    K, M = oracle_mod.assemble_1d(p, m)
    _close(_host(ud), oracle_mod.schwarz_sweep(3, K, M, p, O.s, order, b, u))


def test_cycles_per_iterate_tile_3d(oracle_mod):
    S, O = _tile_pair(oracle_mod, 3, 32)
    b, u0 = synth.coefficients(S.N, 61), synth.initial_guess(S.N, 62)
    ud, bd, uo = _dev(u0), _dev(b), u0.copy()
    for k in range(3):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        rel = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
        assert rel <= TOL, (k, rel)


@pytest.mark.parametrize("precision", [iga2l.MIXED_FP32, iga2l.MIXED_FP32_ALL])
def test_mixed_tile_3d_matches_oracle(oracle_mod, precision):
    """3D mixed TILE form: the oracle's TILE cycle count within one at 1e-8; refined to a
    1e-12 residual, within 1e-8 of the oracle's solution refined the same way."""
    p, m = 3, 32
    S, O = _tile_pair(oracle_mod, p, m, precision)
    f, u0 = synth.coefficients(S.N, 71), synth.initial_guess(S.N, 72)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    b = _host(bd)
    ud = _dev(u0)
    c, _, _, ok = S.solve_load(bd, ud, tol=1e-8, max_cycles=40)
    uo, co, _, _, oko = O.solve(b, u0, tol=1e-8, maxc=40)
    assert ok and oko and abs(c - co) <= 1, (c, co)
    ud = _dev(u0)
    S.solve_load(bd, ud, tol=1e-12, max_cycles=60)
    uo, _, _, _, oko = O.solve(b, u0, tol=1e-12, maxc=60)
    err = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
    assert err <= 1e-8, err


def test_full_size_3d_solves(oracle_mod):
    """128^3 elements, p = 3 (the 3D workload at the size the benchmark times): FP64 and
    mixed solves to 1e-8, each converged solution's residual re-evaluated by the oracle."""
    p, m = 3, 128
    q, g = COLOURING[p]
    O = oracle_mod.Problem(3, p, m, sched=oracle_mod.LATTICE, period=q, stride=g, coarse=oracle_mod.VCYCLE)
    cycles = {}
    for prec in (iga2l.FP64, iga2l.MIXED_FP32):
        S = iga2l.Solver(p, m, dim=3, period=q, stride=g, precision=prec)
        assert S.N == O.N
        f = _dev(synth.coefficients(S.N, 51))
        b = torch.empty_like(f)
        S.rhs_from_coeffs(f, b)
        u0 = synth.initial_guess(S.N, 52)
        ud = _dev(u0)
        cyc, rel, _, ok = S.solve_load(b, ud, tol=1e-8, max_cycles=40)
        assert ok and rel <= 1e-8 and 3 <= cyc <= 20
        bh = _host(b)
        r_end = np.linalg.norm(O.residual(_host(ud), bh))
        r_0 = np.linalg.norm(O.residual(u0, bh))
        assert r_end <= 1.0001e-8 * r_0, (prec, r_end / r_0)
        cycles[prec] = cyc
        S.close()
    assert abs(cycles[iga2l.FP64] - cycles[iga2l.MIXED_FP32]) <= 1
