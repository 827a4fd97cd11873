"""GPU tests of the differentiable solve: the bump source against the oracle's load
vectors, the unrolled backward against the oracle's transposed cycles, and both
gradients (adjoint solve, unrolled 20-cycle backward) against central finite
differences of the same GPU forward map."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402
from paper_2009_01499_gb300.autograd import bump_solve  # noqa: E402

pytestmark = pytest.mark.gpu

W = 0.05


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _oracle_load(oracle_mod, p, m, theta):
    n = m + p - 2
    b = np.zeros(n * n)
    for a, cx, cy in theta:
        gx = oracle_mod.load_1d(p, m, kind=1, par=(cx, W))
        gy = oracle_mod.load_1d(p, m, kind=1, par=(cy, W))
        b += a * np.kron(gy, gx)
    return b


def test_bump_load_and_a_gradient_match_oracle(oracle_mod):
    p, m = 3, 40
    S = iga2l.Solver(p, m, period=7, stride=2)
    theta = synth.bumps(5, 11)
    b = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.bump_load(_dev(theta.ravel()), W, b)
    bo = _oracle_load(oracle_mod, p, m, theta)
    assert np.abs(b.cpu().numpy() - bo).max() <= 1e-12 * np.abs(bo).max()
    lam = synth.uniform_pm1(3, S.N)
    grad = torch.empty(15, dtype=torch.float64, device="cuda")
    S.bump_grad(_dev(theta.ravel()), W, _dev(lam), grad)
    for k, (a, cx, cy) in enumerate(theta):
        gx = oracle_mod.load_1d(p, m, kind=1, par=(cx, W))
        gy = oracle_mod.load_1d(p, m, kind=1, par=(cy, W))
        ref = float(np.dot(lam, np.kron(gy, gx)))
        assert abs(grad[3 * k].item() - ref) <= 1e-12 * np.abs(lam).sum() * np.abs(gx).max() * np.abs(gy).max()


def test_unrolled_backward_matches_oracle(oracle_mod):
    """bbar = sum_k C^T (I - A C^T)^{K-k} ubar with the oracle's transposed cycle."""
    p, m, K = 3, 40, 6
    S = iga2l.Solver(p, m, period=7, stride=2)
    O = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.VCYCLE, period=7, stride=2)
    ubar = synth.uniform_pm1(5, S.N)
    bbar = torch.empty(S.N, dtype=torch.float64, device="cuda")
    S.unrolled_backward(_dev(ubar), K, bbar)
    ub, ref = ubar.copy(), np.zeros(S.N)
    z = np.zeros(S.N)
    for _ in range(K):
        v = O.cycle(z, ub, adjoint=True)
        ref += v
        ub = ub - O.apply_A(v)
    got = bbar.cpu().numpy()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def _loss(S, theta, ut, mode, ncycles=20, tol=1e-13):
    u = bump_solve(theta, S, W, mode=mode, tol=tol, ncycles=ncycles)
    return 0.5 * torch.sum((u - ut) ** 2)


@pytest.mark.parametrize("mode", ["adjoint", "unrolled"])
def test_gradient_against_central_differences(mode):
    p, m, nb = 3, 64, 4
    S = iga2l.Solver(p, m, period=7, stride=2)
    theta0 = synth.bumps(nb, 23)
    ut = _dev(synth.uniform_pm1(24, S.N))
    theta = _dev(theta0.ravel()).requires_grad_(True)
    L = _loss(S, theta, ut, mode)
    L.backward()
    g = theta.grad.cpu().numpy()
    for idx in range(3 * nb):
        h = 1e-5 * max(1.0, abs(theta0.ravel()[idx]))
        tp, tm = theta0.ravel().copy(), theta0.ravel().copy()
        tp[idx] += h
        tm[idx] -= h
        with torch.no_grad():
            Lp = _loss(S, _dev(tp), ut, mode).item()
            Lm = _loss(S, _dev(tm), ut, mode).item()
        fd = (Lp - Lm) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-6 * max(1.0, abs(fd)) + 1e-6 * np.abs(g).max(), (mode, idx, g[idx], fd)


def test_config4_full_size_gradient():
    """p = 3, 512x512 elements, 16 bumps (widths 0.05): the adjoint gradient (solves to a
    1e-12 residual; 1e-13 is below the FP64 rounding floor at this size) against central
    differences of the 40-cycle map, which has converged to that floor and is a smooth
    function of theta; also the unrolled 20-cycle gradient is computed."""
    p, m, nb = 3, 512, 16
    S = iga2l.Solver(p, m, period=7, stride=2)
    theta0 = synth.bumps(nb, synth.BASE_SEED + 5)
    ut = _dev(synth.uniform_pm1(synth.BASE_SEED + 6, S.N))
    theta = _dev(theta0.ravel()).requires_grad_(True)
    L = _loss(S, theta, ut, "adjoint", tol=1e-12)
    L.backward()
    g = theta.grad.cpu().numpy()
    gu = theta.grad.clone()
    theta.grad = None
    Lu = _loss(S, theta, ut, "unrolled")
    Lu.backward()
    assert torch.isfinite(theta.grad).all()
    for idx in (0, 1, 2, 3 * 7 + 1):
        h = 1e-5 * max(1.0, abs(theta0.ravel()[idx]))
        tp, tm = theta0.ravel().copy(), theta0.ravel().copy()
        tp[idx] += h
        tm[idx] -= h
        with torch.no_grad():
            fd = (_loss(S, _dev(tp), ut, "unrolled", ncycles=40).item()
                  - _loss(S, _dev(tm), ut, "unrolled", ncycles=40).item()) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-5 * max(1.0, abs(fd)), (idx, g[idx], fd)
    assert torch.isfinite(gu).all()


def _dense_A_and_mass(oracle_mod, p, m):
    K, M = oracle_mod.assemble_1d(p, m)
    return np.kron(K, M) + np.kron(M, K), np.kron(M, M)


@pytest.mark.parametrize("mode", ["adjoint", "unrolled"])
def test_coefficient_gradient_matches_oracle_and_finite_differences(oracle_mod, mode):
    """dL/df through CoeffSolve (b = (M x M) f, Section 2), L = 0.5 ||u - u_t||^2:
    adjoint mode against the dense (M x M) A^{-1} (u - u_t); unrolled mode against
    (M x M) C_K^T (u_K - u_t) with C_K the oracle's K-cycle map b -> u_K built column by
    column; both against central differences of the GPU map."""
    from paper_2009_01499_gb300.autograd import coeff_solve, load_solve
    p, m, K = 2, 12, 6
    S = iga2l.Solver(p, m, period=5, stride=2, coarse=iga2l.COARSE_EXACT)
    O = oracle_mod.Problem(2, p, m, sched=oracle_mod.LATTICE, coarse=oracle_mod.EXACT, period=5, stride=2)
    N = S.N
    A, MM = _dense_A_and_mass(oracle_mod, p, m)
    f = synth.coefficients(N, 61)
    ut = synth.uniform_pm1(62, N)
    fd = _dev(f).requires_grad_(True)
    u = coeff_solve(fd, S, mode=mode, tol=1e-13, ncycles=K)
    loss = 0.5 * torch.sum((u - _dev(ut)) ** 2)
    loss.backward()
    g = fd.grad.cpu().numpy()
    if mode == "adjoint":
        uo = np.linalg.solve(A, MM @ f)
        ref = MM @ np.linalg.solve(A, uo - ut)
    else:
        CK = np.zeros((N, N))
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            x = np.zeros(N)
            for _ in range(K):
                x = O.cycle(x, e)
            CK[:, j] = x
        uk = CK @ (MM @ f)
        ref = MM @ (CK.T @ (uk - ut))
    assert np.abs(g - ref).max() <= 1e-10 * np.abs(ref).max()
    # central differences of the GPU map along two random directions
    rng = np.random.default_rng(63)
    for _ in range(2):
        v = rng.standard_normal(N)
        h = 1e-6
        lp = float(0.5 * torch.sum((coeff_solve(_dev(f + h * v), S, mode=mode, tol=1e-13, ncycles=K) - _dev(ut)) ** 2))
        lm = float(0.5 * torch.sum((coeff_solve(_dev(f - h * v), S, mode=mode, tol=1e-13, ncycles=K) - _dev(ut)) ** 2))
        fdv = (lp - lm) / (2 * h)
        assert abs(fdv - float(np.dot(g, v))) <= 1e-6 * max(1.0, abs(fdv))
    # the load-vector form gives dL/db = lambda, and (M x M) lambda = dL/df
    bd = torch.empty(N, dtype=torch.float64, device="cuda")
    S.rhs_from_coeffs(_dev(f), bd)
    bd.requires_grad_(True)
    u2 = load_solve(bd, S, mode=mode, tol=1e-13, ncycles=K)
    (0.5 * torch.sum((u2 - _dev(ut)) ** 2)).backward()
    lam = bd.grad.cpu().numpy()
    assert np.abs(MM @ lam - g).max() <= 1e-12 * np.abs(g).max()
    S.close()
