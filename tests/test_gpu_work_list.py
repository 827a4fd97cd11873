"""GPU tests of the work-list TILE sweep (IGA2L_SWEEP_WORK_LIST): the whole TILE sweep of
every problem of a handle in one launch, CTAs claiming (colour group, tile phase, problem,
tile) items in sweep order and each tile waiting (bounded) for the earlier occurrences of
its own and its eight neighbouring tile positions.  Every pair of tiles that touch the same
DOFs keeps the order of one launch per tile phase, so the iterates are bitwise equal to that
form's (which the oracle parity
tests pin); here: sweeps forward and reverse, whole cycles and solves, FP64 and FP32,
colour groups, grids with empty tile phases, batches with problems masked mid-solve, and
the bounded wait running out."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3), 6: (11, 4)}


def _pair(p, m, **kw):
    q, g = COLOURING[p]
    A = iga2l.Solver(p, m, period=q, stride=g, schedule=iga2l.SCHED_TILE, **kw)
    B = iga2l.Solver(p, m, period=q, stride=g, schedule=iga2l.SCHED_TILE, sweep=iga2l.SWEEP_WORK_LIST, **kw)
    return A, B


def _vec(n, seed):
    return torch.tensor(synth.uniform_pm1(seed, n), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("p,m,groups", [(2, 100, 1), (3, 108, 2), (4, 92, 1), (5, 132, 1), (6, 100, 4), (6, 88, 0),
                                        (2, 12, 1), (3, 16, 1)])
def test_fp64_sweeps_and_cycles_bitwise_equal(p, m, groups):
    A, B = _pair(p, m, tile_groups=groups)
    b, u = _vec(A.N, 7 * p + m), _vec(A.N, 9 * p + m)
    for reverse in (False, True):
        ua, ub = u.clone(), u.clone()
        A.schwarz_sweep(ua, b, reverse=reverse)
        B.schwarz_sweep(ub, b, reverse=reverse)
        torch.cuda.synchronize()
        assert torch.equal(ua, ub), reverse
        assert not torch.equal(ua, u)
    ua, ub = u.clone(), u.clone()
    for _ in range(2):
        A.cycle(ua, b)
        B.cycle(ub, b)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)


@pytest.mark.parametrize("precision", [iga2l.MIXED_FP32, iga2l.MIXED_FP32_ALL])
@pytest.mark.parametrize("p,m", [(2, 128), (3, 96), (5, 100)])
def test_mixed_solves_bitwise_equal(p, m, precision):
    A, B = _pair(p, m, precision=precision)
    f = torch.tensor(synth.coefficients(A.N, 40 + p), device="cuda")
    u0 = torch.tensor(synth.initial_guess(A.N, 41 + p), device="cuda")
    ua, ub = u0.clone(), u0.clone()
    ca, ra, _, oka = A.solve(f, ua, tol=1e-8)
    cb, rb, _, okb = B.solve(f, ub, tol=1e-8)
    assert oka and okb and ca == cb and ra == rb
    assert torch.equal(ua, ub)
    us, vs = _vec(A.N, 3).float(), _vec(A.N, 4).float()
    ua32, ub32 = us.clone(), us.clone()
    A.schwarz_sweep_f32(ua32, vs, reverse=True)
    B.schwarz_sweep_f32(ub32, vs, reverse=True)
    torch.cuda.synchronize()
    assert torch.equal(ua32, ub32)


@pytest.mark.parametrize("precision", [iga2l.FP64, iga2l.MIXED_FP32])
def test_batch_bitwise_equal_with_masked_problems(precision):
    p, m, nb = 3, 64, 7
    q, g = COLOURING[p]
    kw = dict(nbatch=nb, period=q, stride=g, precision=precision, schedule=iga2l.SCHED_TILE, tile_groups=2)
    A = iga2l.Solver(p, m, **kw)
    B = iga2l.Solver(p, m, sweep=iga2l.SWEEP_WORK_LIST, **kw)
    N = A.N
    f = torch.tensor(np.concatenate([synth.coefficients(N, 500 + k) for k in range(nb)]), device="cuda")
    u0 = torch.tensor(np.concatenate([synth.initial_guess(N, 600 + k) for k in range(nb)]), device="cuda")
    # problem 1 starts converged (zero data), problem 4 from a guess close to its solution,
    # so problems leave the batch at different cycles
    f[N:2 * N] = 0.0
    u0[N:2 * N] = 0.0
    ref = u0.clone()
    A.solve_batch(f, ref, tol=1e-12)
    u0[4 * N:5 * N] = ref[4 * N:5 * N] + 1e-6 * u0[4 * N:5 * N]
    ua, ub = u0.clone(), u0.clone()
    ca, ra, oka = A.solve_batch(f, ua, tol=1e-8)
    cb, rb, okb = B.solve_batch(f, ub, tol=1e-8)
    assert oka and okb and list(ca) == list(cb) and list(ra) == list(rb)
    assert ca[1] == 0 and ca[4] < max(ca)
    assert torch.equal(ua, ub)


def test_withheld_tile_counts_time_out_and_context_survives():
    p, m = 2, 64
    q, g = COLOURING[p]
    S = iga2l.Solver(p, m, period=q, stride=g, schedule=iga2l.SCHED_TILE, sweep=iga2l.SWEEP_WORK_LIST,
                     test_flags=iga2l.TEST_WITHHOLD_PROGRESS, wait_budget_cycles=20000)
    f = torch.tensor(synth.coefficients(S.N, 5), device="cuda")
    u = torch.tensor(synth.initial_guess(S.N, 6), device="cuda")
    with pytest.raises(iga2l.IgaError) as ei:
        S.solve(f, u, tol=1e-8, max_cycles=2)
    assert ei.value.code == iga2l.ERR_DEVICE_TIMEOUT
    S.close()
    torch.cuda.synchronize()
    A, B = _pair(p, m)
    ua = torch.tensor(synth.initial_guess(A.N, 6), device="cuda")
    ub = ua.clone()
    ca, _, _, oka = A.solve(f, ua, tol=1e-8)
    cb, _, _, okb = B.solve(f, ub, tol=1e-8)
    assert oka and okb and ca == cb and torch.equal(ua, ub)


def test_work_list_needs_the_tile_schedule():
    with pytest.raises(iga2l.IgaError) as ei:
        iga2l.Solver(3, 32, sweep=iga2l.SWEEP_WORK_LIST)
    assert ei.value.code == iga2l.ERR_UNSUPPORTED
