"""GPU parity for the higher degrees of the paper's experiments (Table 4 runs p = 2..8):
p = 6 with 5x5 Schwarz blocks, p = 7, 8 with 7x7 blocks (Sections 4.3, 5.1), against the
FP64 oracle.  Bars: cycle counts equal to the oracle's; mixed forms within 1e-8 of the
FP64 oracle after refinement; FP64 per iterate within max(1e-12, 8 kappa eps), kappa the
largest condition number of the degree's Schwarz blocks (the GPU applies precomputed
block inverses, the oracle Cholesky-solves each block: two FP64 evaluations that differ by
~kappa eps; kappa is 4e2 at p = 5, so 1e-12 there, but 1.3e3 / 2.0e4 / 6.9e4 at
p = 6 / 7 / 8).  The TILE schedule is compiled for blocks up to 5x5 (p <= 6)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
# m >= 4p + 4, even; sizes with ragged tiles and colours
SIZES = {6: 50, 7: 40, 8: 44}


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _pair(oracle_mod, p, m, sched="lattice", precision=iga2l.FP64, coarse="vcycle"):
    sg = iga2l.SCHED_TILE if sched == "tile" else iga2l.SCHED_LATTICE
    cg = iga2l.COARSE_VCYCLE if coarse == "vcycle" else iga2l.COARSE_EXACT
    S = iga2l.Solver(p, m, schedule=sg, precision=precision, coarse=cg)
    so = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    co = oracle_mod.VCYCLE if coarse == "vcycle" else oracle_mod.EXACT
    O = oracle_mod.Problem(2, p, m, sched=so, tile=S.tile or 32, coarse=co, period=S.period, stride=S.stride,
                           groups=S.tile_groups)
    assert S.N == O.N and S.block_side == O.s
    assert (S.period, S.stride) == oracle_mod.DEFAULT_COLOURING[p]
    return S, O


def block_kappa(oracle_mod, p, m):
    """Largest 2-norm condition number of the Schwarz blocks A_B = K_B (x) M_B + M_B (x) K_B
    (clipped s x s blocks; the interior block and every boundary class)."""
    K, M = oracle_mod.assemble_1d(p, m)
    n, s = K.shape[0], oracle_mod.block_size(p)
    r, L = (s - 1) // 2, p - 1 + (s - 1) // 2
    worst = 0.0
    for cy in list(range(L + 1)) + [n // 2]:
        for cx in list(range(L + 1)) + [n // 2]:
            xs = [x for x in range(cx - r, cx + r + 1) if 0 <= x < n]
            ys = [y for y in range(cy - r, cy + r + 1) if 0 <= y < n]
            A = np.kron(K[np.ix_(ys, ys)], M[np.ix_(xs, xs)]) + np.kron(M[np.ix_(ys, ys)], K[np.ix_(xs, xs)])
            worst = max(worst, np.linalg.cond(A))
    return worst


def fp64_tol(oracle_mod, p, m):
    return max(TOL, 8.0 * block_kappa(oracle_mod, p, m) * np.finfo(float).eps / 2)


def _close(got, ref, tol=TOL):
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err <= tol, f"max rel diff {err:.3e}"


@pytest.mark.parametrize("p", [6, 7, 8])
def test_residual_and_apply_high_p(oracle_mod, p):
    m = SIZES[p]
    S, O = _pair(oracle_mod, p, m)
    b, u = synth.coefficients(S.N, 10 + p), synth.initial_guess(S.N, 11 + p)
    d = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.residual(_dev(u), _dev(b), d)
    _close(_host(d), O.residual(u, b))


@pytest.mark.parametrize("p,sched", [(6, "lattice"), (6, "tile"), (7, "lattice"), (8, "lattice")])
@pytest.mark.parametrize("reverse", [False, True])
def test_schwarz_sweep_high_p(oracle_mod, p, sched, reverse):
    m = SIZES[p]
    S, O = _pair(oracle_mod, p, m, sched=sched)
    b, u = synth.coefficients(S.N, 20 + p), synth.initial_guess(S.N, 21 + p)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b), reverse=reverse)
    kind = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    _, order, _ = oracle_mod.schedule(2, S.n, O.s, p, kind, S.tile or 32, S.period, S.stride, S.tile_groups)
    if reverse:
        order = order[::-1].copy()
    K, M = oracle_mod.assemble_1d(p, m)
    _close(_host(ud), oracle_mod.schwarz_sweep(2, K, M, p, O.s, order, b, u), fp64_tol(oracle_mod, p, m))


@pytest.mark.parametrize("p,sched", [(6, "lattice"), (6, "tile"), (7, "lattice"), (8, "lattice")])
def test_cycles_per_iterate_high_p(oracle_mod, p, sched):
    m = SIZES[p]
    S, O = _pair(oracle_mod, p, m, sched=sched)
    f, u0 = synth.coefficients(S.N, 30 + p), synth.initial_guess(S.N, 31 + p)
    K, M = oracle_mod.assemble_1d(p, m)
    b = (M @ f.reshape(S.n, S.n) @ M.T).ravel()
    ud, bd, uo = _dev(u0), _dev(b), u0.copy()
    tol = fp64_tol(oracle_mod, p, m)
    for k in range(3):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        rel = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
        assert rel <= tol, f"cycle {k + 1}: {rel:.3e} > {tol:.1e}"


@pytest.mark.parametrize("p", [6, 7, 8])
def test_solve_counts_and_mixed_high_p(oracle_mod, p):
    """Cycle counts to 1e-8 equal the oracle's (FP64); both mixed forms take the same count
    within one cycle and, refined to a 1e-15 residual reduction, are within 1e-8 of the FP64
    oracle's solution refined the same way.  (The discrete operator's condition number grows
    quickly with p; from the random start, which is ~10^4 times the solution, the oracle's
    own solutions at 1e-12 and 1e-14 differ by 2e-7 (p = 6) to 1e-6 (p = 8), and at 1e-15
    they are settled to ~3e-9, so the comparison is made there.)"""
    m = 64
    S, O = _pair(oracle_mod, p, m)
    f, u0 = synth.coefficients(S.N, 40 + p), synth.initial_guess(S.N, 41 + p)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    b = _host(bd)
    ud = _dev(u0)
    cyc, rel, hist, ok = S.solve_load(bd, ud, tol=1e-8, max_cycles=40)
    uo, cyc_o, rel_o, hist_o, ok_o = O.solve(b, u0, tol=1e-8, maxc=40)
    assert ok and ok_o and cyc == cyc_o
    assert np.linalg.norm(_host(ud) - uo) <= fp64_tol(oracle_mod, p, m) * np.linalg.norm(uo)
    ref, _, _, _, ok_r = O.solve(b, u0, tol=1e-15, maxc=200)
    assert ok_r
    modes = [(iga2l.MIXED_FP32, "tile" if p <= 6 else "lattice"),
             (iga2l.MIXED_FP32_ALL, "tile" if p <= 6 else "lattice")]
    for prec, sched in modes:
        X, _ = _pair(oracle_mod, p, m, sched=sched, precision=prec)
        um = _dev(u0)
        c, _, _, okm = X.solve_load(bd, um, tol=1e-8, max_cycles=40)
        if sched == "lattice":
            assert okm and abs(c - cyc_o) <= 1, (prec, c, cyc_o)
        um = _dev(u0)
        c, _, _, okm = X.solve_load(bd, um, tol=1e-15, max_cycles=200)
        assert okm
        err = np.linalg.norm(_host(um) - ref) / np.linalg.norm(ref)
        assert err <= 1e-8, (prec, err)


def test_tile_rejected_for_7x7_blocks():
    with pytest.raises(iga2l.IgaError) as ei:
        iga2l.Solver(7, 40, schedule=iga2l.SCHED_TILE)
    assert ei.value.code == iga2l.ERR_UNSUPPORTED
    for p in (6, 7):   # the tensor-core form: single 2D problems, LATTICE, p <= 5
        with pytest.raises(iga2l.IgaError) as ei:
            iga2l.Solver(p, 40, precision=iga2l.MIXED_TF32)
        assert ei.value.code == iga2l.ERR_UNSUPPORTED


@pytest.mark.parametrize("p", [6, 7, 8])
def test_full_size_high_degree_solves(oracle_mod, p):
    """1024x1024 elements (the size the benchmark times for p = 6..8): FP64 and mixed solves
    to 1e-8 with the default colouring, each converged solution's residual re-evaluated by
    the oracle; the mixed form's cycle count within one of the FP64 form's."""
    m = 1024
    O = None
    cycles = {}
    for prec in (iga2l.FP64, iga2l.MIXED_FP32):
        S = iga2l.Solver(p, m, precision=prec)
        if O is None:
            O = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE,
                                   period=S.period, stride=S.stride)
        f = _dev(synth.coefficients(S.N, 60 + p))
        b = torch.empty_like(f)
        S.rhs_from_coeffs(f, b)
        u0 = synth.initial_guess(S.N, 70 + p)
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
