"""Thin ctypes binding of the C ABI in include/iga2l.h.

Argument marshalling only: every step of the solver runs in libiga2l.so's CUDA
kernels.  Vectors are torch float64 CUDA tensors (contiguous, x fastest);
streams default to torch's current stream.  If the library cannot be loaded
the binding raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_NONFINITE, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
FP64, MIXED_FP32, MIXED_FP32_ALL, MIXED_TF32 = 0, 1, 2, 3
SCHED_LATTICE, SCHED_TILE = 1, 2
COARSE_EXACT, COARSE_VCYCLE = 0, 1
RHS_COEFFS, RHS_IS_LOAD = 0, 1
SWEEP_AUTO, SWEEP_PER_COLOUR, SWEEP_PERSISTENT, SWEEP_WORK_LIST = 0, 1, 2, 3
TEST_SKIP_OPERATOR_COPY, TEST_WITHHOLD_PROGRESS, TEST_GUARD_ALLOCS = 1, 2, 4

# Every exported symbol of include/iga2l.h.
EXPORTS = (
    "iga2l_default_options", "iga2l_assemble", "iga2l_num_dofs", "iga2l_apply_A",
    "iga2l_residual", "iga2l_schwarz_sweep", "iga2l_schwarz_sweep_reverse", "iga2l_restrict",
    "iga2l_prolong_add", "iga2l_coarse_solve", "iga2l_cycle", "iga2l_cycle_adjoint",
    "iga2l_solve", "iga2l_adjoint_solve", "iga2l_rhs_from_coeffs", "iga2l_get_bands",
    "iga2l_host_bands", "iga2l_host_restriction", "iga2l_destroy", "iga2l_strerror",
    "iga2l_last_error", "iga2l_kernel_launches", "iga2l_residual_norm2_noalloc",
    "iga2l_cycles", "iga2l_unrolled_backward", "iga2l_bump_load", "iga2l_bump_grad",
    "iga2l_assemble_batch", "iga2l_solve_batch", "iga2l_schedule_info", "iga2l_solve_load",
    "iga2l_schwarz_sweep_f32", "iga2l_fma_peak", "iga2l_guard_check",
)


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int), ("tile", ctypes.c_int),
                ("period", ctypes.c_int), ("stride", ctypes.c_int), ("coarse", ctypes.c_int),
                ("block_side", ctypes.c_int), ("max_cycles", ctypes.c_int), ("graphs", ctypes.c_int),
                ("rhs", ctypes.c_int), ("tile_groups", ctypes.c_int), ("sweep", ctypes.c_int),
                ("test_flags", ctypes.c_int), ("wait_budget_cycles", ctypes.c_longlong)]


class IgaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"iga2l error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None
_vp, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
_ip, _llp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong)


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libiga2l.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libiga2l.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        sig = {
            "iga2l_default_options": (None, [ctypes.POINTER(Options)]),
            "iga2l_assemble": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
            "iga2l_num_dofs": (ctypes.c_int, [_vp, _llp, _ip, _llp, _ip]),
            "iga2l_schedule_info": (ctypes.c_int, [_vp, _ip, _ip, _ip, _ip, _ip, _ip]),
            "iga2l_apply_A": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_residual": (ctypes.c_int, [_vp, _vp, _vp, _vp, _dp, _vp]),
            "iga2l_schwarz_sweep": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_schwarz_sweep_reverse": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_restrict": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_schwarz_sweep_f32": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
            "iga2l_prolong_add": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_coarse_solve": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_cycle": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_cycle_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _ip, _dp,
                                           _dp, _vp]),
            "iga2l_solve_load": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _ip, _dp,
                                                _dp, _vp]),
            "iga2l_adjoint_solve": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp,
                                                   _ip, _dp, _vp]),
            "iga2l_rhs_from_coeffs": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
            "iga2l_get_bands": (ctypes.c_int, [_vp, _dp, _dp]),
            "iga2l_host_bands": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, _dp]),
            "iga2l_host_restriction": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp]),
            "iga2l_destroy": (None, [_vp]),
            "iga2l_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "iga2l_last_error": (ctypes.c_char_p, []),
            "iga2l_kernel_launches": (ctypes.c_longlong, []),
            "iga2l_guard_check": (ctypes.c_int, [_vp, _llp]),
            "iga2l_fma_peak": (ctypes.c_int, [ctypes.c_int, _dp, _vp]),
            "iga2l_cycles": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
            "iga2l_assemble_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(Options), ctypes.POINTER(_vp)]),
            "iga2l_solve_batch": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_int, _vp, _ip, _dp, _vp]),
            "iga2l_unrolled_backward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
            "iga2l_bump_load": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp]),
            "iga2l_bump_grad": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_double, _vp, _vp, _vp]),
            "iga2l_residual_norm2_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                                            _vp, _vp, _vp, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc, allow_not_converged=False):
    if rc == OK or (allow_not_converged and rc == NOT_CONVERGED):
        return rc
    lib = load()
    raise IgaError(rc, f"{lib.iga2l_strerror(rc).decode()}: {lib.iga2l_last_error().decode()}")


def _ptr(t, dtype="float64", numel=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != getattr(torch, dtype) or not t.is_contiguous():
        raise TypeError(f"expected a contiguous {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} entries, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def kernel_launches() -> int:
    """Kernels launched by libiga2l.so in this process so far."""
    return int(load().iga2l_kernel_launches())


def fma_peak(kind: int, stream=None) -> float:
    """Measured FMA-pipe throughput (GFLOP/s): kind 0 FP64, 1 FP32, 2 packed FP32 pairs."""
    g = ctypes.c_double(0.0)
    _check(load().iga2l_fma_peak(int(kind), ctypes.byref(g), _stream(stream)))
    return g.value


def default_options(**kw) -> Options:
    o = Options()
    load().iga2l_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


def host_bands(p: int, m: int):
    """Library's 1D band rows (host setup code, no GPU): K, M as n x (2p+1)."""
    n, w = m + p - 2, 2 * p + 1
    K = np.zeros(n * w)
    M = np.zeros(n * w)
    _check(load().iga2l_host_bands(p, m, K.ctypes.data_as(_dp), M.ctypes.data_as(_dp)))
    return K.reshape(n, w), M.reshape(n, w)


def host_restriction(p: int, m: int):
    """Library's dense 1D aggressive restriction (host setup code, no GPU)."""
    n, nc = m + p - 2, m // 2 - 1
    R = np.zeros(nc * n)
    _check(load().iga2l_host_restriction(p, m, R.ctypes.data_as(_dp)))
    return R.reshape(nc, n)


def residual_norm2_noalloc(p, n, Kb, Mb, u, b, d, norm2, stream=None):
    """Handle-free defect d = b - A u and ||d||^2 (device scalar) for callers that
    cannot allocate device memory; Kb, Mb are device copies of the 1D band rows.
    The library allocates nothing for this call (see include/iga2l.h)."""
    _check(load().iga2l_residual_norm2_noalloc(
        int(p), int(n), _ptr(Kb, numel=n * (2 * p + 1)), _ptr(Mb, numel=n * (2 * p + 1)),
        _ptr(u, numel=n * n), _ptr(b, numel=n * n), _ptr(d, numel=n * n) if d is not None else None,
        _ptr(norm2, numel=1), _stream(stream)))


class Solver:
    """Handle of one assembled problem (degree p, m elements per axis, dimension dim),
    or with nbatch > 1 of a batch of 2D problems sharing (p, m, options)."""

    def __init__(self, p: int, m: int, dim: int = 2, nbatch: int = 1, batch: bool = False, **options):
        self._lib = load()
        self.options = default_options(**options)
        h = _vp()
        if nbatch > 1 or batch:
            _check(self._lib.iga2l_assemble_batch(p, m, nbatch, ctypes.byref(self.options), ctypes.byref(h)))
        else:
            _check(self._lib.iga2l_assemble(p, m, dim, ctypes.byref(self.options), ctypes.byref(h)))
        self._h = h
        self.p, self.m, self.dim, self.nbatch = p, m, dim, nbatch
        nt, na, nct, nca = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_int()
        _check(self._lib.iga2l_num_dofs(h, ctypes.byref(nt), ctypes.byref(na), ctypes.byref(nct),
                                        ctypes.byref(nca)))
        self.N, self.n, self.Nc, self.nc = nt.value, na.value, nct.value, nca.value
        self.NB, self.NcB = self.N * nbatch, self.Nc * nbatch   # vector lengths seen by the ABI
        sc, q, g, t, s, tg = (ctypes.c_int() for _ in range(6))
        _check(self._lib.iga2l_schedule_info(h, ctypes.byref(sc), ctypes.byref(q), ctypes.byref(g), ctypes.byref(t),
                                             ctypes.byref(s), ctypes.byref(tg)))
        self.schedule, self.period, self.stride, self.tile, self.block_side = sc.value, q.value, g.value, t.value, s.value
        self.tile_groups = tg.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.iga2l_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- single steps -------------------------------------------------------
    def apply_A(self, u, y, stream=None):
        _check(self._lib.iga2l_apply_A(self._h, _ptr(u, numel=self.NB), _ptr(y, numel=self.NB),
                                       _stream(stream)))

    def residual(self, u, b, d=None, want_norm=False, stream=None):
        nrm = ctypes.c_double(0.0)
        _check(self._lib.iga2l_residual(self._h, _ptr(u, numel=self.NB), _ptr(b, numel=self.NB),
                                        _ptr(d, numel=self.NB) if d is not None else None,
                                        ctypes.byref(nrm) if want_norm else None, _stream(stream)))
        return nrm.value if want_norm else None

    def schwarz_sweep(self, u, b, reverse=False, stream=None):
        fn = self._lib.iga2l_schwarz_sweep_reverse if reverse else self._lib.iga2l_schwarz_sweep
        _check(fn(self._h, _ptr(u, numel=self.NB), _ptr(b, numel=self.NB), _stream(stream)))

    def schwarz_sweep_f32(self, u, b, reverse=False, stream=None):
        """The inner cycle's FP32 Schwarz step on float32 vectors (mixed-precision handles)."""
        _check(self._lib.iga2l_schwarz_sweep_f32(self._h, _ptr(u, "float32", self.N), _ptr(b, "float32", self.N),
                                                 int(bool(reverse)), _stream(stream)))

    def restrict(self, d, dc, stream=None):
        _check(self._lib.iga2l_restrict(self._h, _ptr(d, numel=self.NB), _ptr(dc, numel=self.NcB),
                                        _stream(stream)))

    def prolong_add(self, ec, u, stream=None):
        _check(self._lib.iga2l_prolong_add(self._h, _ptr(ec, numel=self.NcB), _ptr(u, numel=self.NB),
                                           _stream(stream)))

    def coarse_solve(self, dc, ec, stream=None):
        _check(self._lib.iga2l_coarse_solve(self._h, _ptr(dc, numel=self.NcB), _ptr(ec, numel=self.NcB),
                                            _stream(stream)))

    def cycle(self, u, b, adjoint=False, stream=None):
        fn = self._lib.iga2l_cycle_adjoint if adjoint else self._lib.iga2l_cycle
        _check(fn(self._h, _ptr(u, numel=self.NB), _ptr(b, numel=self.NB), _stream(stream)))

    def rhs_from_coeffs(self, f, b, stream=None):
        _check(self._lib.iga2l_rhs_from_coeffs(self._h, _ptr(f, numel=self.NB), _ptr(b, numel=self.NB),
                                               _stream(stream)))

    # --- solves -------------------------------------------------------------
    def _solve(self, fn, rhs, u, tol, max_cycles, stream):
        cap = max_cycles if max_cycles > 0 else self.options.max_cycles
        hist = np.zeros(cap)
        cyc, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = _check(fn(self._h, _ptr(rhs, numel=self.N), float(tol), cap, _ptr(u, numel=self.N),
                       ctypes.byref(cyc), ctypes.byref(rel), hist.ctypes.data_as(_dp), _stream(stream)),
                    allow_not_converged=True)
        return cyc.value, rel.value, hist[: cyc.value].copy(), rc == OK

    def solve(self, f, u, tol=1e-8, max_cycles=0, stream=None):
        """Solve A u = b with b = (f, phi_i) of the source given by its B-spline coefficients f
        (or b itself on a handle built with rhs=RHS_IS_LOAD); cycles in place on u.
        Returns (cycles, relres, history, converged)."""
        return self._solve(self._lib.iga2l_solve, f, u, tol, max_cycles, stream)

    def solve_load(self, b, u, tol=1e-8, max_cycles=0, stream=None):
        """Solve A u = b for a load vector b given directly; as solve() otherwise."""
        return self._solve(self._lib.iga2l_solve_load, b, u, tol, max_cycles, stream)

    def adjoint_solve(self, g, lam, tol=1e-8, max_cycles=0, stream=None):
        cyc, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        rc = _check(self._lib.iga2l_adjoint_solve(self._h, _ptr(g, numel=self.N), float(tol),
                                                  int(max_cycles), _ptr(lam, numel=self.N),
                                                  ctypes.byref(cyc), ctypes.byref(rel), _stream(stream)),
                    allow_not_converged=True)
        return cyc.value, rel.value, rc == OK

    def solve_batch(self, rhs, u, tol=1e-8, max_cycles=0, stream=None):
        """All problems of a batch handle to tol; rhs holds every problem's coefficient vector f
        (or load vector b with rhs=RHS_IS_LOAD).  Returns (cycles[], relres[], converged)."""
        nb = self.nbatch
        cyc = (ctypes.c_int * nb)()
        rel = np.zeros(nb)
        rc = _check(self._lib.iga2l_solve_batch(self._h, _ptr(rhs, numel=nb * self.N), float(tol), int(max_cycles),
                                                _ptr(u, numel=nb * self.N), cyc, rel.ctypes.data_as(_dp),
                                                _stream(stream)), allow_not_converged=True)
        return np.array(cyc[:], dtype=np.int64), rel, rc == OK

    def cycles(self, u, b, ncycles, stream=None):
        _check(self._lib.iga2l_cycles(self._h, _ptr(u, numel=self.NB), _ptr(b, numel=self.NB), int(ncycles),
                                      _stream(stream)))

    def unrolled_backward(self, ubar, ncycles, bbar, stream=None):
        _check(self._lib.iga2l_unrolled_backward(self._h, _ptr(ubar, numel=self.N), int(ncycles),
                                                 _ptr(bbar, numel=self.N), _stream(stream)))

    def bump_load(self, theta, width, b, stream=None):
        nb = theta.numel() // 3
        _check(self._lib.iga2l_bump_load(self._h, nb, _ptr(theta, numel=3 * nb), float(width),
                                         _ptr(b, numel=self.N), _stream(stream)))

    def bump_grad(self, theta, width, bbar, grad, stream=None):
        nb = theta.numel() // 3
        _check(self._lib.iga2l_bump_grad(self._h, nb, _ptr(theta, numel=3 * nb), float(width),
                                         _ptr(bbar, numel=self.N), _ptr(grad, numel=3 * nb), _stream(stream)))

    def bands(self):
        w = 2 * self.p + 1
        K = np.zeros(self.n * w)
        M = np.zeros(self.n * w)
        _check(self._lib.iga2l_get_bands(self._h, K.ctypes.data_as(_dp), M.ctypes.data_as(_dp)))
        return K.reshape(self.n, w), M.reshape(self.n, w)

    def guard_check(self) -> int:
        """Bytes of the handle's guard zones that changed (handles assembled with
        test_flags=TEST_GUARD_ALLOCS); synchronises the device."""
        c = ctypes.c_longlong(0)
        _check(self._lib.iga2l_guard_check(self._h, ctypes.byref(c)))
        return c.value
