"""GPU tests of batched solves: a batch handle gives each problem exactly the iterates,
cycle count and residual of a single solve (converged problems are masked on the
device), in FP64 and in the mixed form; the multi-group solver of uneven (p, m)
problems matches single solves per problem."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402
from paper_2009_01499_gb300.batch import BatchedSolver  # noqa: E402

pytestmark = pytest.mark.gpu

COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2)}


@pytest.mark.parametrize("precision,sched", [(0, 1), (1, 2)])
def test_batch_equals_single_solves(precision, sched):
    p, m, nb = 3, 64, 6
    q, g = COLOURING[p]
    B = iga2l.Solver(p, m, nbatch=nb, period=q, stride=g, precision=precision, schedule=sched,
                     rhs=iga2l.RHS_IS_LOAD)
    S = iga2l.Solver(p, m, period=q, stride=g, precision=precision, schedule=sched)
    f = torch.tensor(np.concatenate([synth.coefficients(S.N, 100 + k) for k in range(nb)]), device="cuda")
    # problem 2 gets a zero right-hand side and guess: done before any cycle
    f[2 * S.N:3 * S.N] = 0.0
    b = torch.empty_like(f)
    B.rhs_from_coeffs(f, b)
    u0 = torch.tensor(np.concatenate([synth.initial_guess(S.N, 200 + k) for k in range(nb)]), device="cuda")
    u0[2 * S.N:3 * S.N] = 0.0
    ub = u0.clone()
    cyc, rel, ok = B.solve_batch(b, ub, tol=1e-8)
    assert ok and cyc[2] == 0
    for k in range(nb):
        sl = slice(k * S.N, (k + 1) * S.N)
        us = u0[sl].clone()
        bs = b[sl].clone()
        c1, r1, _, ok1 = S.solve_load(bs, us, tol=1e-8)
        assert ok1 and c1 == cyc[k], (k, c1, cyc[k])
        assert torch.equal(us, ub[sl]), k
        if c1:
            assert abs(r1 - rel[k]) <= 1e-12 * r1


def test_uneven_groups_match_single_solves():
    problems = [(2, 64), (3, 32), (2, 64), (4, 48), (3, 32), (2, 128), (4, 48), (3, 64)]
    BS = BatchedSolver(problems, precision=iga2l.MIXED_FP32, autotune=True)
    f = [torch.tensor(synth.coefficients((m + p - 2) ** 2, 300 + i), device="cuda") for i, (p, m) in enumerate(problems)]
    u0 = [torch.tensor(synth.initial_guess((m + p - 2) ** 2, 400 + i), device="cuda") for i, (p, m) in enumerate(problems)]
    b = BS.rhs_from_coeffs(BS.pack(f))
    u = BS.pack(u0)
    cycles, relres, ok = BS.solve(BS.pack(f), u, tol=1e-8)   # coefficients f (the default)
    torch.cuda.synchronize()
    assert ok
    ub = BS.unpack(u)
    bb = BS.unpack(b)
    for g in BS.groups:
        p, m = g["p"], g["m"]
        q, gg = COLOURING[p]
        S = iga2l.Solver(p, m, period=q, stride=gg, precision=iga2l.MIXED_FP32, schedule=g["schedule"],
                         tile_groups=g["tile_groups"])
        for i in g["members"]:
            us = u0[i].clone()
            c1, r1, _, ok1 = S.solve_load(bb[i].clone(), us, tol=1e-8)
            assert ok1 and c1 == cycles[i] and torch.equal(us, ub[i]), (i, c1, cycles[i])
        S.close()
    BS.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_concurrent_handles_match_sequential(precision):
    """Independent handles solving at once on their own streams and host threads (as the
    benchmark's concurrent step does) give exactly the sequential iterates."""
    import threading
    probs = [(2, 96), (3, 80), (4, 88), (5, 72)]
    solvers, bs, u0s = [], [], []
    for i, (p, m) in enumerate(probs):
        S = iga2l.Solver(p, m, precision=precision,
                         schedule=iga2l.SCHED_TILE if precision else iga2l.SCHED_LATTICE)
        f = torch.tensor(synth.coefficients(S.N, 300 + i), device="cuda")
        b = torch.empty_like(f)
        S.rhs_from_coeffs(f, b)
        solvers.append(S)
        bs.append(b)
        u0s.append(torch.tensor(synth.initial_guess(S.N, 400 + i), device="cuda"))
    seq = []
    for S, b, u0 in zip(solvers, bs, u0s):
        u = u0.clone()
        c, rel, _, ok = S.solve_load(b, u, tol=1e-8)
        assert ok
        seq.append((u, c, rel))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in probs]
    us = [u0.clone() for u0 in u0s]
    torch.cuda.synchronize()
    out = [None] * len(probs)

    def run(k):
        out[k] = solvers[k].solve_load(bs[k], us[k], tol=1e-8, stream=streams[k])

    threads = [threading.Thread(target=run, args=(k,)) for k in range(len(probs))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    for k in range(len(probs)):
        c, rel, _, ok = out[k]
        assert ok and c == seq[k][1] and rel == seq[k][2], k
        assert torch.equal(us[k], seq[k][0]), k


def test_full_size_batch_residuals(oracle_mod):
    """The 256-problem workload (m in {64, 128, 256, 512}, p in {2, 3, 4}, seeded; 26.7M
    DOFs), mixed precision with autotuned schedules and concurrent groups: every problem
    converges, and its residual re-evaluated by the oracle meets the 1e-8 rule."""
    nprob = 256
    z = synth.splitmix64(synth.BASE_SEED + 4, 2 * nprob)
    ms = np.array([64, 128, 256, 512])[(z[0::2] % np.uint64(4)).astype(int)]
    ps = np.array([2, 3, 4])[(z[1::2] % np.uint64(3)).astype(int)]
    problems = [(int(p), int(m)) for p, m in zip(ps, ms)]
    BS = BatchedSolver(problems, precision=iga2l.MIXED_FP32, autotune=True)
    f = [torch.tensor(synth.coefficients((m + p - 2) ** 2, 1000 + i), device="cuda") for i, (p, m) in enumerate(problems)]
    u0 = [torch.tensor(synth.initial_guess((m + p - 2) ** 2, 2000 + i), device="cuda")
          for i, (p, m) in enumerate(problems)]
    b = BS.rhs_from_coeffs(BS.pack(f))
    u = BS.pack(u0)
    cycles, relres, ok = BS.solve(BS.pack(f), u, tol=1e-8)
    assert ok and max(cycles) <= 20 and max(relres) <= 1e-8
    bs, us = BS.unpack(b), BS.unpack(u)
    oracles = {}
    for i, (p, m) in enumerate(problems):
        if (p, m) not in oracles:
            oracles[(p, m)] = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE)
        O = oracles[(p, m)]
        bh = bs[i].cpu().numpy()
        r_end = np.linalg.norm(O.residual(us[i].cpu().numpy(), bh))
        r_0 = np.linalg.norm(O.residual(u0[i].cpu().numpy(), bh))
        assert r_end <= 1.0001e-8 * r_0, (i, p, m, r_end / r_0)
    BS.close()
