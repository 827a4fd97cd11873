"""The oracle's OpenMP build (the threaded CPU baseline) gives the sequential oracle's
results bit for bit: its parallel loops split only independent work (the blocks of one
Schwarz colour, the points of one Gauss-Seidel sub-lattice, stencil and transfer
outputs) and never a sum."""
import numpy as np
import pytest

from paper_2009_01499_gb300 import synth


@pytest.mark.parametrize("dim,p,m,sched,coarse", [
    (2, 2, 32, 1, 1), (2, 5, 40, 1, 1), (2, 3, 42, 2, 1), (2, 4, 24, 0, 0), (3, 2, 16, 1, 1), (3, 3, 12, 1, 0)])
def test_threaded_oracle_is_bit_identical(oracle_mod, dim, p, m, sched, coarse):
    A = oracle_mod.Problem(dim, p, m, sched=sched, tile=21 if p == 3 else 32, coarse=coarse)
    B = oracle_mod.Problem(dim, p, m, sched=sched, tile=21 if p == 3 else 32, coarse=coarse, threads=4)
    assert A.threads == 1 and B.threads == 4
    b = synth.coefficients(A.N, 5)
    u0 = synth.initial_guess(A.N, 6)
    ua, ub = A.cycle(u0, b), B.cycle(u0, b)
    assert np.array_equal(ua, ub)
    assert np.array_equal(A.cycle(ua, b, adjoint=True), B.cycle(ub, b, adjoint=True))
    assert np.array_equal(A.residual(ua, b), B.residual(ub, b))
    _, ca, ra, ha, _ = A.solve(b, u0, tol=1e-6, maxc=12)
    _, cb, rb, hb, _ = B.solve(b, u0, tol=1e-6, maxc=12)
    assert ca == cb and np.array_equal(ha, hb)
