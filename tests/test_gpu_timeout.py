"""GPU test of the bounded device waits: the tensor-core colour kernel's wait for the
bulk copy of its block operator gives up after options.wait_budget_cycles and the solve
reports IGA2L_ERR_DEVICE_TIMEOUT.

The failure is made without any fault: IGA2L_TEST_SKIP_OPERATOR_COPY makes the kernel
not issue that copy at all, so no asynchronous copy and no MMA is ever in flight; the
wait runs out, the kernel records it in its status word, skips its blocks, releases its
tensor memory and returns.  The results of that call are discarded, and a normal solve
on the same device right after it must still be correct."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_missing_operator_copy_times_out_and_context_survives(oracle_mod):
    p, m = 2, 48
    S = iga2l.Solver(p, m, precision=iga2l.MIXED_TF32, schedule=iga2l.SCHED_LATTICE,
                     test_flags=iga2l.TEST_SKIP_OPERATOR_COPY, wait_budget_cycles=20000)
    f = torch.tensor(synth.coefficients(S.N, 5), device="cuda")
    u = torch.tensor(synth.initial_guess(S.N, 6), device="cuda")
    with pytest.raises(iga2l.IgaError) as ei:
        S.solve(f, u, tol=1e-8, max_cycles=2)
    assert ei.value.code == iga2l.ERR_DEVICE_TIMEOUT
    S.close()
    torch.cuda.synchronize()
    # the same form without the test flag converges, and matches the oracle's cycle count
    T = iga2l.Solver(p, m, precision=iga2l.MIXED_TF32, schedule=iga2l.SCHED_LATTICE)
    u = torch.tensor(synth.initial_guess(T.N, 6), device="cuda")
    cyc, rel, _, ok = T.solve(f, u, tol=1e-8, max_cycles=40)
    O = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE,
                           period=T.period, stride=T.stride)
    K, M = oracle_mod.assemble_1d(p, m)
    fh = f.cpu().numpy()
    b = (M @ fh.reshape(T.n, T.n) @ M.T).ravel()
    _, cyc_o, _, _, ok_o = O.solve(b, synth.initial_guess(T.N, 6), tol=1e-8, maxc=40)
    assert ok and ok_o and cyc == cyc_o
    r = np.linalg.norm(O.residual(u.cpu().numpy(), b)) / np.linalg.norm(O.residual(synth.initial_guess(T.N, 6), b))
    assert r <= 1.0001e-8
    T.close()


def test_withheld_progress_times_out_and_context_survives():
    """The persistent sweep: CTA 0 never raises its progress counter, so its neighbours'
    bounded waits give up, every CTA leaves its colour loop, and the solve reports the
    timeout; a normal solve right after it converges."""
    p, m = 3, 64
    S = iga2l.Solver(p, m, precision=iga2l.MIXED_FP32, sweep=iga2l.SWEEP_PERSISTENT,
                     test_flags=iga2l.TEST_WITHHOLD_PROGRESS, wait_budget_cycles=200000)
    f = torch.tensor(synth.coefficients(S.N, 15), device="cuda")
    u = torch.tensor(synth.initial_guess(S.N, 16), device="cuda")
    with pytest.raises(iga2l.IgaError) as ei:
        S.solve(f, u, tol=1e-8, max_cycles=2)
    assert ei.value.code == iga2l.ERR_DEVICE_TIMEOUT
    S.close()
    torch.cuda.synchronize()
    T = iga2l.Solver(p, m, precision=iga2l.MIXED_FP32, sweep=iga2l.SWEEP_PERSISTENT)
    u = torch.tensor(synth.initial_guess(T.N, 16), device="cuda")
    cyc, rel, _, ok = T.solve(f, u, tol=1e-8, max_cycles=40)
    assert ok and rel <= 1e-8
    T.close()


def test_wait_budget_is_validated():
    with pytest.raises(iga2l.IgaError) as ei:
        iga2l.Solver(2, 48, wait_budget_cycles=-1)
    assert ei.value.code == iga2l.ERR_INVALID_ARG
