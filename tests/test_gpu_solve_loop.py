"""GPU: the device-driven solve (one CUDA graph whose WHILE node repeats the cycle and its
convergence check on the device) against the host-driven loop (graphs off: one norm read
back per cycle).  Both take the stopping decision with the same arithmetic
(rel = sqrt(||r_k||^2) / ||r_0||, Section 5's rule), so cycle counts, residual histories
and iterates agree bit for bit, including at the cycle cap and in the mixed-precision
and adjoint solves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3)}


def _pair(p, m, **kw):
    q, g = COLOURING[p]
    A = iga2l.Solver(p, m, period=q, stride=g, graphs=1, **kw)
    B = iga2l.Solver(p, m, period=q, stride=g, graphs=0, **kw)
    return A, B


def _vecs(S, seed):
    f = torch.tensor(synth.coefficients(S.N, seed), device="cuda")
    b = torch.empty_like(f)
    S.rhs_from_coeffs(f, b)
    u0 = torch.tensor(synth.initial_guess(S.N, seed + 1), device="cuda")
    return b, u0


@pytest.mark.parametrize("p,m,prec,sched", [
    (2, 40, iga2l.FP64, iga2l.SCHED_LATTICE),
    (5, 48, iga2l.FP64, iga2l.SCHED_LATTICE),
    (3, 64, iga2l.MIXED_FP32, iga2l.SCHED_TILE),
    (4, 62, iga2l.MIXED_FP32_ALL, iga2l.SCHED_LATTICE),
])
def test_device_loop_equals_host_loop(p, m, prec, sched):
    A, B = _pair(p, m, precision=prec, schedule=sched)
    b, u0 = _vecs(A, 300 + p)
    ua, ub = u0.clone(), u0.clone()
    ca, ra, ha, oka = A.solve_load(b, ua, tol=1e-9, max_cycles=50)
    cb, rb, hb, okb = B.solve_load(b, ub, tol=1e-9, max_cycles=50)
    assert oka and okb and ca == cb and ra == rb
    assert np.array_equal(ha, hb) and torch.equal(ua, ub)
    assert ha[-1] <= 1e-9 < ha[-2]


def test_cycle_cap_stops_the_device_loop():
    A, B = _pair(3, 48)
    b, u0 = _vecs(A, 311)
    ua, ub = u0.clone(), u0.clone()
    ca, ra, ha, oka = A.solve_load(b, ua, tol=1e-30, max_cycles=3)
    cb, rb, hb, okb = B.solve_load(b, ub, tol=1e-30, max_cycles=3)
    assert not oka and not okb and ca == cb == 3 and len(ha) == 3
    assert np.array_equal(ha, hb) and torch.equal(ua, ub)
    # the next solve on the same graph starts from a fresh control block
    ua2 = u0.clone()
    ca2, _, ha2, ok2 = A.solve_load(b, ua2, tol=1e-8, max_cycles=40)
    assert ok2 and ca2 > 3 and np.array_equal(ha2[:3], ha)


def test_adjoint_device_loop_equals_host_loop():
    A, B = _pair(2, 36)
    g, _ = _vecs(A, 321)
    la, lb = torch.zeros_like(g), torch.zeros_like(g)
    ca, ra, oka = A.adjoint_solve(g, la, tol=1e-10)
    cb, rb, okb = B.adjoint_solve(g, lb, tol=1e-10)
    assert oka and okb and ca == cb and ra == rb and torch.equal(la, lb)


def test_device_loop_counts_its_kernels():
    A, _ = _pair(2, 32)
    b, u0 = _vecs(A, 331)
    u = u0.clone()
    A.solve_load(b, u, tol=1e-8)          # builds the graph
    u = u0.clone()
    n0 = iga2l.kernel_launches()
    cyc, _, _, ok = A.solve_load(b, u, tol=1e-8)
    per_cycle = (iga2l.kernel_launches() - n0 - 1) / cyc   # minus the initial residual
    assert ok and per_cycle == int(per_cycle) and per_cycle > 25


@pytest.mark.parametrize("precision,sched", [(iga2l.FP64, iga2l.SCHED_LATTICE), (iga2l.MIXED_FP32, iga2l.SCHED_TILE)])
def test_batched_device_loop_equals_host_loop(precision, sched):
    """Batch handles: the WHILE loop stops once no problem is active (k_batch_check)."""
    p, m, nb = 2, 48, 5
    q, g = COLOURING[p]
    A = iga2l.Solver(p, m, nbatch=nb, period=q, stride=g, precision=precision, schedule=sched, graphs=1)
    B = iga2l.Solver(p, m, nbatch=nb, period=q, stride=g, precision=precision, schedule=sched, graphs=0,
                     rhs=iga2l.RHS_IS_LOAD)
    N = (m + p - 2) ** 2
    f = torch.tensor(np.concatenate([synth.coefficients(N, 400 + k) for k in range(nb)]), device="cuda")
    b = torch.empty_like(f)
    A.rhs_from_coeffs(f, b)
    u0 = torch.tensor(np.concatenate([synth.initial_guess(N, 500 + k) for k in range(nb)]), device="cuda")
    ua, ub = u0.clone(), u0.clone()
    ca, ra, oka = A.solve_batch(f, ua, tol=1e-9)   # coefficients: b formed by the library
    cb, rb, okb = B.solve_batch(b, ub, tol=1e-9)   # the load vector given directly
    assert oka and okb and list(ca) == list(cb) and np.array_equal(ra, rb) and torch.equal(ua, ub)
    # at a cycle cap every problem stops after exactly that many cycles
    ua, ub = u0.clone(), u0.clone()
    ca, ra, oka = A.solve_batch(f, ua, tol=1e-30, max_cycles=2)
    cb, rb, okb = B.solve_batch(b, ub, tol=1e-30, max_cycles=2)
    assert not oka and not okb and list(ca) == list(cb) == [2] * nb and torch.equal(ua, ub)
