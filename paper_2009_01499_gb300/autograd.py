"""torch.autograd bindings of the differentiable two-level solve.

``CoeffSolve.apply(f, solver, mode, tol, ncycles)`` returns the control points u of
A u = b, b = (f, phi_i) = (M (x) M) f (Section 2), for a source given by its B-spline
coefficients f; backward gives dL/df = (M (x) M) lambda with lambda = dL/db from the
adjoint solve (or the unrolled backward).  ``LoadSolve.apply(b, ...)`` takes the load
vector b itself and returns dL/db = lambda.

``BumpSolve.apply(theta, solver, width, mode, tol, ncycles)`` returns u(theta), the
control points of the 2D Poisson solution for the source
f = sum_k a_k exp(-|x - c_k|^2 / (2 width^2)), theta = [(a_k, cx_k, cy_k)].

Forward: b = (f, phi) by the library's bump kernels, then either
  mode "adjoint":  a solve to ``tol`` (Algorithm 1 cycles), or
  mode "unrolled": ``ncycles`` cycles from u = 0 (the truncated iteration itself).
Backward (all in the library's kernels, FP64):
  "adjoint":  lambda = A^{-1} ubar by the transposed-cycle solve (A is symmetric),
  "unrolled": bbar = sum_k C^T (I - A C^T)^{K-k} ubar, exact for the truncated
              iteration; the cycle is affine in u, so no forward state is stored
              (the only nonlinear stage, theta -> b, is recomputed from theta),
then dL/dtheta from bbar by the bump-gradient kernel.  This module only
allocates tensors and calls the C ABI.
"""
from __future__ import annotations

import torch

from . import iga2l


def _forward(solver, b, mode, tol, ncycles):
    if mode not in ("adjoint", "unrolled"):
        raise ValueError("mode must be 'adjoint' or 'unrolled'")
    u = torch.zeros_like(b)
    if mode == "adjoint":
        cyc, rel, _, ok = solver.solve_load(b, u, tol=tol, max_cycles=200)
        if not ok:
            raise RuntimeError(f"forward solve did not reach {tol:g} (rel {rel:.3e})")
    else:
        solver.cycles(u, b, ncycles)
    return u


def _load_adjoint(solver, ubar, mode, tol, ncycles):
    """dL/db for dL/du = ubar: the adjoint solve or the unrolled backward."""
    ubar = ubar.contiguous().to(torch.float64)
    bbar = torch.zeros(solver.N, dtype=torch.float64, device=ubar.device)
    if mode == "adjoint":
        cyc, rel, ok = solver.adjoint_solve(ubar, bbar, tol=tol, max_cycles=200)
        if not ok:
            raise RuntimeError(f"adjoint solve did not reach {tol:g} (rel {rel:.3e})")
    else:
        solver.unrolled_backward(ubar, ncycles, bbar)
    return bbar


class LoadSolve(torch.autograd.Function):
    """u = A^{-1} b (adjoint mode) or ncycles cycles from u = 0 (unrolled mode)."""

    @staticmethod
    def forward(ctx, b, solver, mode="adjoint", tol=1e-12, ncycles=20):
        u = _forward(solver, b.detach().contiguous(), mode, tol, ncycles)
        ctx.solver, ctx.mode, ctx.tol, ctx.ncycles = solver, mode, tol, ncycles
        return u

    @staticmethod
    def backward(ctx, ubar):
        return _load_adjoint(ctx.solver, ubar, ctx.mode, ctx.tol, ctx.ncycles), None, None, None, None


class CoeffSolve(torch.autograd.Function):
    """u for the source with B-spline coefficients f: b = (M (x) M) f formed by the library."""

    @staticmethod
    def forward(ctx, f, solver, mode="adjoint", tol=1e-12, ncycles=20):
        fd = f.detach().contiguous()
        b = torch.empty_like(fd)
        solver.rhs_from_coeffs(fd, b)
        u = _forward(solver, b, mode, tol, ncycles)
        ctx.solver, ctx.mode, ctx.tol, ctx.ncycles = solver, mode, tol, ncycles
        return u

    @staticmethod
    def backward(ctx, ubar):
        S = ctx.solver
        bbar = _load_adjoint(S, ubar, ctx.mode, ctx.tol, ctx.ncycles)
        fbar = torch.empty_like(bbar)
        S.rhs_from_coeffs(bbar, fbar)     # (M (x) M)^T = M (x) M
        return fbar, None, None, None, None


class BumpSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, solver, width, mode="adjoint", tol=1e-12, ncycles=20):
        if mode not in ("adjoint", "unrolled"):
            raise ValueError("mode must be 'adjoint' or 'unrolled'")
        th = theta.detach().contiguous()
        b = torch.empty(solver.N, dtype=torch.float64, device=th.device)
        solver.bump_load(th, width, b)
        u = torch.zeros_like(b)
        if mode == "adjoint":
            cyc, rel, _, ok = solver.solve_load(b, u, tol=tol, max_cycles=200)
            if not ok:
                raise RuntimeError(f"forward solve did not reach {tol:g} (rel {rel:.3e})")
        else:
            solver.cycles(u, b, ncycles)
        ctx.save_for_backward(th)
        ctx.solver, ctx.width, ctx.mode, ctx.tol, ctx.ncycles = solver, width, mode, tol, ncycles
        return u

    @staticmethod
    def backward(ctx, ubar):
        (th,) = ctx.saved_tensors
        S = ctx.solver
        ubar = ubar.contiguous().to(torch.float64)
        bbar = torch.zeros(S.N, dtype=torch.float64, device=ubar.device)
        if ctx.mode == "adjoint":
            cyc, rel, ok = S.adjoint_solve(ubar, bbar, tol=ctx.tol, max_cycles=200)
            if not ok:
                raise RuntimeError(f"adjoint solve did not reach {ctx.tol:g} (rel {rel:.3e})")
        else:
            S.unrolled_backward(ubar, ctx.ncycles, bbar)
        grad = torch.empty_like(th)
        S.bump_grad(th, ctx.width, bbar, grad)
        return grad, None, None, None, None, None


def coeff_solve(f, solver: "iga2l.Solver", mode="adjoint", tol=1e-12, ncycles=20):
    """u(f) with dL/df = (M x M) lambda through the library's adjoint or unrolled backward."""
    return CoeffSolve.apply(f, solver, mode, tol, ncycles)


def load_solve(b, solver: "iga2l.Solver", mode="adjoint", tol=1e-12, ncycles=20):
    """u(b) with dL/db = lambda through the library's adjoint or unrolled backward."""
    return LoadSolve.apply(b, solver, mode, tol, ncycles)


def bump_solve(theta, solver: "iga2l.Solver", width=0.05, mode="adjoint", tol=1e-12, ncycles=20):
    """u(theta) with gradients through the library's adjoint or unrolled backward."""
    return BumpSolve.apply(theta, solver, width, mode, tol, ncycles)
