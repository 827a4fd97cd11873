"""GPU parity on tiny 2D grids, down to every Schwarz block and every stencil row being a
boundary one: in place of a memory checker, the boundary paths of every kernel on their
own.

The library accepts even m >= max(4, p + 1), i.e. n = m + p - 2 >= 2p - 1 DOFs per axis:
  * with n < 2L + 1 (L = p - 1 + r) no block centre is interior;
  * with n < 4p - 1 no stencil row is;
  * the second level is then solved directly.
Per degree the sizes are the smallest grid, a middle one and the one below the former
limit 4p + 4.  Against the FP64 oracle, with the library's default colouring:
  * residual and A u element by element to 1e-12 of the max;
  * LATTICE and TILE sweeps (forward and reverse) to the block-condition FP64 bar;
  * transfers and the second-level solve;
  * three cycles per iterate;
  * cycle counts to 1e-8;
  * the mixed forms: cycle counts, and after refinement within 1e-8 of the oracle's
    solution.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12
TINY = {2: (4, 6, 10), 3: (4, 8, 14), 4: (6, 10, 18), 5: (6, 10, 22), 6: (8, 14, 26), 7: (8, 14, 30),
        8: (10, 16, 34)}
CASES = [(p, m) for p, ms in TINY.items() for m in ms]
SMALLEST = [(p, ms[0]) for p, ms in TINY.items()]


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _close(got, ref, tol=TOL):
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)
    assert err <= tol, f"max rel diff {err:.3e} > {tol:.1e}"


def _pair(oracle_mod, p, m, sched="lattice", precision=iga2l.FP64, **kw):
    sg = iga2l.SCHED_TILE if sched == "tile" else iga2l.SCHED_LATTICE
    S = iga2l.Solver(p, m, schedule=sg, precision=precision, **kw)
    so = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    O = oracle_mod.Problem(2, p, m, sched=so, tile=S.tile or 32, coarse=oracle_mod.VCYCLE, period=S.period,
                           stride=S.stride, groups=S.tile_groups)
    assert S.N == O.N and S.Nc == O.Nc and S.block_side == O.s
    return S, O


def _fp64_tol(oracle_mod, p, m):
    """1e-12, or 8 kappa eps / 2 with kappa the largest condition number of the grid's
    (clipped) Schwarz blocks, every centre of the tiny grid taken."""
    K, M = oracle_mod.assemble_1d(p, m)
    n, s = K.shape[0], oracle_mod.block_size(p)
    r = (s - 1) // 2
    worst = 0.0
    for cy in range(n):
        ys = [y for y in range(cy - r, cy + r + 1) if 0 <= y < n]
        for cx in range(cy, n):   # A_B for (cx, cy) and (cy, cx) are similar
            xs = [x for x in range(cx - r, cx + r + 1) if 0 <= x < n]
            A = np.kron(K[np.ix_(ys, ys)], M[np.ix_(xs, xs)]) + np.kron(M[np.ix_(ys, ys)], K[np.ix_(xs, xs)])
            worst = max(worst, np.linalg.cond(A))
    return max(TOL, 8.0 * worst * np.finfo(float).eps / 2)


def test_smallest_grids_have_no_interior_block_or_row(oracle_mod):
    """The smallest accepted grid of every degree is all boundary: n < 2L + 1 and n < 4p - 1."""
    for p, m in SMALLEST:
        n, s = m + p - 2, oracle_mod.block_size(p)
        L = p - 1 + (s - 1) // 2
        assert n >= 2 * p - 1 and n < 2 * L + 1 and n < 4 * p - 1, (p, m)


@pytest.mark.parametrize("p,m", CASES)
def test_tiny_residual_and_apply(oracle_mod, p, m):
    S, O = _pair(oracle_mod, p, m)
    f, u = synth.coefficients(S.N, 900 + p), synth.initial_guess(S.N, 901 + p)
    d = torch.empty(S.N, dtype=torch.float64, device="cuda")
    nrm = S.residual(_dev(u), _dev(f), d, want_norm=True)
    ref = O.residual(u, f)
    _close(_host(d), ref)
    assert abs(nrm - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref)   # the call returns ||d||
    y = torch.empty_like(d)
    S.apply_A(_dev(u), y)
    _close(_host(y), O.apply_A(u))


@pytest.mark.parametrize("p,m", CASES)
@pytest.mark.parametrize("sched", ["lattice", "tile"])
@pytest.mark.parametrize("reverse", [False, True])
def test_tiny_schwarz_sweep(oracle_mod, p, m, sched, reverse):
    if sched == "tile" and p > 6:
        pytest.skip("the TILE schedule is compiled for p <= 6")
    S, O = _pair(oracle_mod, p, m, sched)
    b, u = synth.coefficients(S.N, 910 + p), synth.initial_guess(S.N, 911 + p)
    ud = _dev(u)
    S.schwarz_sweep(ud, _dev(b), reverse=reverse)
    kind = oracle_mod.TILE if sched == "tile" else oracle_mod.LATTICE
    _, order, _ = oracle_mod.schedule(2, S.n, O.s, p, kind, S.tile or 32, S.period, S.stride, S.tile_groups)
    if reverse:
        order = order[::-1].copy()
    K, M = oracle_mod.assemble_1d(p, m)
    _close(_host(ud), oracle_mod.schwarz_sweep(2, K, M, p, O.s, order, b, u), _fp64_tol(oracle_mod, p, m))


@pytest.mark.parametrize("p,m", CASES)
def test_tiny_transfers_and_coarse_solve(oracle_mod, p, m):
    S, O = _pair(oracle_mod, p, m)
    d, u = synth.coefficients(S.N, 920 + p), synth.initial_guess(S.N, 921 + p)
    dc = torch.empty(S.Nc, dtype=torch.float64, device="cuda")
    S.restrict(_dev(d), dc)
    dco = O.restrict(d)
    _close(_host(dc), dco)
    ec = torch.empty_like(dc)
    S.coarse_solve(_dev(dco), ec)
    eco = O.coarse_solve(dco)
    _close(_host(ec), eco)
    ud = _dev(u)
    S.prolong_add(_dev(eco), ud)
    _close(_host(ud), O.prolong_add(eco, u))


@pytest.mark.parametrize("p,m", CASES)
@pytest.mark.parametrize("sched", ["lattice", "tile"])
def test_tiny_cycles_per_iterate_and_solve(oracle_mod, p, m, sched):
    if sched == "tile" and p > 6:
        pytest.skip("the TILE schedule is compiled for p <= 6")
    S, O = _pair(oracle_mod, p, m, sched)
    f, u0 = synth.coefficients(S.N, 930 + p), synth.initial_guess(S.N, 931 + p)
    K, M = oracle_mod.assemble_1d(p, m)
    b = (M @ f.reshape(S.n, S.n) @ M.T).ravel()
    ud, bd, uo = _dev(u0), _dev(b), u0.copy()
    tol = _fp64_tol(oracle_mod, p, m)
    for k in range(3):
        S.cycle(ud, bd)
        uo = O.cycle(uo, b)
        rel = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
        assert rel <= tol, f"cycle {k + 1}: {rel:.3e} > {tol:.1e}"
    ud = _dev(u0)
    c, rel, _, ok = S.solve(_dev(f), ud, tol=1e-8, max_cycles=60)
    _, co, _, _, oko = O.solve(b, u0, tol=1e-8, maxc=60)
    assert ok and oko and c == co, (c, co)


MIXED = [(iga2l.MIXED_FP32, "lattice", {"sweep": iga2l.SWEEP_PER_COLOUR}),
         (iga2l.MIXED_FP32, "lattice", {}),
         (iga2l.MIXED_FP32, "tile", {}),
         (iga2l.MIXED_FP32, "tile", {"sweep": iga2l.SWEEP_WORK_LIST}),
         (iga2l.MIXED_FP32_ALL, "tile", {})]


@pytest.mark.parametrize("p,m", CASES)
@pytest.mark.parametrize("precision,sched,kw", MIXED)
def test_tiny_mixed_refinement(oracle_mod, p, m, precision, sched, kw):
    """Cycle counts to 1e-8 within one of the FP64 oracle's in the same order; refined to a
    1e-12 residual, within 1e-8 of the oracle's solution."""
    if sched == "tile" and p > 6:
        pytest.skip("the TILE schedule is compiled for p <= 6")
    S, O = _pair(oracle_mod, p, m, sched, precision, **kw)
    f, u0 = synth.coefficients(S.N, 940 + p), synth.initial_guess(S.N, 941 + p)
    bd = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    b = _host(bd)
    ud = _dev(u0)
    c, _, _, ok = S.solve_load(bd, ud, tol=1e-8, max_cycles=60)
    _, co, _, _, oko = O.solve(b, u0, tol=1e-8, maxc=60)
    assert ok and oko and abs(c - co) <= 1, (c, co)
    ud = _dev(u0)
    c, _, _, ok = S.solve_load(bd, ud, tol=1e-12, max_cycles=80)
    uo, co, _, _, oko = O.solve(b, u0, tol=1e-12, maxc=80)
    assert ok and oko
    err = np.linalg.norm(_host(ud) - uo) / np.linalg.norm(uo)
    assert err <= 1e-8, err


def test_tiny_grid_rules():
    """Below the 2D minimum, and for the forms built for grids with interior blocks, the
    handle is refused with an error."""
    with pytest.raises(iga2l.IgaError):
        iga2l.Solver(8, 8)            # n = 14 < 2p - 1
    with pytest.raises(iga2l.IgaError):
        iga2l.Solver(2, 2)            # no 2h level
    with pytest.raises(iga2l.IgaError):
        iga2l.Solver(3, 14, dim=3)    # 3D: m >= 4p + 4
    with pytest.raises(iga2l.IgaError):
        iga2l.Solver(3, 14, precision=iga2l.MIXED_TF32)
    with pytest.raises(iga2l.IgaError):
        iga2l.Solver(3, 14, precision=iga2l.MIXED_FP32, sweep=iga2l.SWEEP_PERSISTENT)
    # AUTO on a small grid: one launch per colour instead of the persistent sweep
    S = iga2l.Solver(8, 34, precision=iga2l.MIXED_FP32)
    u = torch.zeros(S.N, dtype=torch.float64, device="cuda")
    S.cycle(u, torch.ones_like(u))
    torch.cuda.synchronize()
    assert torch.isfinite(u).all()
