"""Plain FP64 CPU oracle of the two-level IGA method (arXiv 2009.01499).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package.  The product library never
imports, links or calls it, and it shares no code with the CUDA path.

The arithmetic lives in plain C (``spline.c``, ``operators.c``), compiled with
gcc at ``-O2 -ffp-contract=off`` (no fused multiply-add contraction, no
fast-math), so x86_64 and aarch64 hosts give bit-identical results.  This
module only builds the shared object and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SO_OMP = os.path.join(_BUILD, "liboracle_omp.so")
_SRCS = [os.path.join(_HERE, f) for f in ("spline.c", "operators.c")]
_HDR = os.path.join(_HERE, "iga_oracle.h")
_lock = threading.Lock()
_lib = None

LEX, LATTICE, TILE = 0, 1, 2
EXACT, VCYCLE = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` and its OpenMP build
    ``liboracle_omp.so`` (if stale)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRCS + [_HDR])
    for so, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if not force and os.path.exists(so) and os.path.getmtime(so) >= newest:
            continue
        tmp = so + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", *extra,
               "-shared", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, so)
    return _SO


_lib_omp = None


def _load(threaded: bool = False):
    """The plain oracle, or its OpenMP build (identical results) when threaded."""
    global _lib, _lib_omp
    with _lock:
        if threaded and _lib_omp is not None:
            return _lib_omp
        if not threaded and _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_SO_OMP if threaded else _SO)
        sig = {
            "or_knots": (None, [ctypes.c_int, ctypes.c_int, _dp]),
            "or_basis_eval": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]),
            "or_gauss": (None, [ctypes.c_int, _dp, _dp]),
            "or_assemble_1d": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
            "or_mixed_mass_1d": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
            "or_load_1d": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, _dp]),
            "or_embed_p1": (None, [ctypes.c_int, _dp]),
            "or_restriction_1d": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
            "or_block_size": (ctypes.c_int, [ctypes.c_int]),
            "or_apply_A": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]),
            "or_schedule": (ctypes.c_int, [ctypes.c_int] * 8 + [_ip, _ip]),
            "or_schwarz_sweep": (None, [ctypes.c_int] * 4 + [_dp, _dp, _ip, _dp, _dp]),
            "or_cholesky": (ctypes.c_int, [ctypes.c_int, _dp]),
            "or_cholesky_solve": (None, [ctypes.c_int, _dp, _dp, _dp]),
            "or_setup": (ctypes.c_void_p, [ctypes.c_int] * 10),
            "or_setup_grouped": (ctypes.c_void_p, [ctypes.c_int] * 11),
            "or_setup_plow": (ctypes.c_void_p, [ctypes.c_int] * 12),
            "or_embed_spline": (None, [ctypes.c_int, ctypes.c_int, _dp]),
            "or_restriction_plow": (None, [ctypes.c_int] * 4 + [_dp]),
            "or_schedule_grouped": (ctypes.c_int, [ctypes.c_int] * 9 + [_ip, _ip]),
            "or_free": (None, [ctypes.c_void_p]),
            "or_n": (ctypes.c_int, [ctypes.c_void_p]),
            "or_nc": (ctypes.c_int, [ctypes.c_void_p]),
            "or_ndofs": (ctypes.c_longlong, [ctypes.c_void_p]),
            "or_residual": (None, [ctypes.c_void_p, _dp, _dp, _dp]),
            "or_norm2": (ctypes.c_double, [ctypes.c_longlong, _dp]),
            "or_smooth": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_restrict": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_prolong_add": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_coarse_solve": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_vcycle_level": (None, [ctypes.c_void_p, ctypes.c_int, _dp, _dp]),
            "or_cycle": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_cycle_adjoint": (None, [ctypes.c_void_p, _dp, _dp]),
            "or_solve": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _dp, _ip, _dp, _dp]),
        }
        sig["or_set_threads"] = (None, [ctypes.c_int])
        sig["or_threads"] = (ctypes.c_int, [])
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if threaded:
            _lib_omp = lib
        else:
            _lib = lib
        return lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _i(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ip)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---- Section 2.1: splines ----------------------------------------------------

def knots(p: int, m: int) -> np.ndarray:
    xi = np.empty(2 * p + m + 1)
    _load().or_knots(p, m, _d(xi))
    return xi


def basis_eval(p: int, m: int, x: float):
    """Full basis N_1..N_{m+p} and derivatives at x (Cox-de Boor)."""
    N = np.empty(m + p)
    dN = np.empty(m + p)
    _load().or_basis_eval(p, m, float(x), _d(N), _d(dN))
    return N, dN


def gauss(npts: int):
    x = np.empty(npts)
    w = np.empty(npts)
    _load().or_gauss(npts, _d(x), _d(w))
    return x, w


def assemble_1d(p: int, m: int, full: bool = False):
    nf = m + p if full else m + p - 2
    K = np.empty((nf, nf))
    M = np.empty((nf, nf))
    _load().or_assemble_1d(p, m, int(full), _d(K), _d(M))
    return K, M


def mixed_mass_1d(p: int, plow: int, m: int) -> np.ndarray:
    Mx = np.empty((m + plow - 2, m + p - 2))
    _load().or_mixed_mass_1d(p, plow, m, _d(Mx))
    return Mx


def load_1d(p: int, m: int, kind: int = 0, par=(0.0, 1.0), nq: int | None = None) -> np.ndarray:
    """g_i = int f1 N_i; kind 0: sin(pi x); kind 1: Gaussian exp(-(x-c)^2/(2w^2)), par=(c, w)."""
    nq = p + 3 if nq is None else nq
    g = np.empty(m + p - 2)
    pa = _f64(par)
    _load().or_load_1d(p, m, kind, _d(pa), nq, _d(g))
    return g


def embed_p1(mc: int) -> np.ndarray:
    S = np.empty((2 * mc - 1, mc - 1))
    _load().or_embed_p1(mc, _d(S))
    return S


def restriction_1d(p: int, m: int, aggressive: bool = True) -> np.ndarray:
    rows = m // 2 - 1 if aggressive else m - 1
    R = np.empty((rows, m + p - 2))
    _load().or_restriction_1d(p, m, int(aggressive), _d(R))
    return R


def embed_spline(plow: int, mc: int) -> np.ndarray:
    """Degree-plow embedding of the 2h space into the h space (or_embed_spline)."""
    S = np.empty((2 * mc + plow - 2, mc + plow - 2))
    _load().or_embed_spline(plow, mc, _d(S))
    return S


def restriction_plow(p: int, plow: int, m: int, aggressive: bool = True) -> np.ndarray:
    rows = (m // 2 if aggressive else m) + plow - 2
    R = np.empty((rows, m + p - 2))
    _load().or_restriction_plow(p, plow, m, int(aggressive), _d(R))
    return R


def block_size(p: int) -> int:
    return _load().or_block_size(p)


# ---- Section 3.1.1 -------------------------------------------------------------

def apply_A(dim: int, K: np.ndarray, M: np.ndarray, u: np.ndarray, w: int) -> np.ndarray:
    n = K.shape[0]
    K = _f64(K); M = _f64(M); u = _f64(u)
    y = np.empty(n ** dim)
    _load().or_apply_A(dim, n, w, _d(K), _d(M), _d(u), _d(y))
    return y


# Colour period q and stride g per degree used by the tests and the benchmark
# (this project's choice; see or_schedule in iga_oracle.h).
DEFAULT_COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3), 6: (11, 4), 7: (14, 5), 8: (17, 4)}


def default_colouring(p: int, s: int):
    return DEFAULT_COLOURING.get(p, (s + p, 1))


def schedule(dim: int, n: int, s: int, p: int, kind: int, tile: int = 0,
             period: int = 0, stride: int = 0, groups: int = 1):
    """Colour of every block centre and the processing order (groups: colour groups of
    the TILE order, or_schedule_grouped)."""
    if kind != LEX and period <= 0:
        period, stride = default_colouring(p, s)
    N = n ** dim
    colour = np.empty(N, dtype=np.int32)
    order = np.empty(N, dtype=np.int32)
    nc = _load().or_schedule_grouped(dim, n, s, p, kind, tile, period, stride, groups, _i(colour), _i(order))
    if nc < 0:
        raise ValueError("bad schedule arguments")
    return colour, order, nc


def schwarz_sweep(dim: int, K, M, w: int, s: int, order: np.ndarray, b, u) -> np.ndarray:
    n = K.shape[0]
    K = _f64(K); M = _f64(M); b = _f64(b)
    u = _f64(u).copy()
    order = np.ascontiguousarray(order, dtype=np.int32)
    _load().or_schwarz_sweep(dim, n, w, s, _d(K), _d(M), _i(order), _d(b), _d(u))
    return u


def cholesky(A: np.ndarray) -> np.ndarray:
    L = _f64(A).copy()
    if _load().or_cholesky(L.shape[0], _d(L)) != 0:
        raise np.linalg.LinAlgError("not SPD")
    return L


def cholesky_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    L = _f64(L); b = _f64(b)
    x = np.empty_like(b)
    _load().or_cholesky_solve(L.shape[0], _d(L), _d(b), _d(x))
    return x


# ---- Algorithm 1 -----------------------------------------------------------------

class Problem:
    """Oracle two-level solver for one (dim, p, m) problem.

    sched: LEX / LATTICE / TILE (tile = T), colour period q / stride g;
    coarse: EXACT or VCYCLE; aggressive: degree-1 second level on 2h
    (Section 3.3) or on h (Section 3.1).
    """

    def __init__(self, dim: int, p: int, m: int, s: int = 0, sched: int = TILE,
                 tile: int = 32, coarse: int = VCYCLE, aggressive: bool = True,
                 period: int = 0, stride: int = 0, groups: int = 1, plow: int = 1, threads: int = 1):
        """threads > 1: the OpenMP build of the oracle with that many threads (results
        identical to the sequential oracle)."""
        lib = _load(threaded=threads > 1)
        if threads > 1:
            lib.or_set_threads(int(threads))
        self.threads = lib.or_threads()
        self._lib = lib
        s_eff = s if s > 0 else block_size(p)
        if period <= 0:
            period, stride = default_colouring(p, s_eff)
        self.period, self.stride = period, stride
        self._h = lib.or_setup_plow(dim, p, m, s, sched, tile, period, stride, groups, coarse,
                                    int(aggressive), plow)
        self.groups, self.plow = groups, plow
        if not self._h:
            raise ValueError(f"oracle setup failed for dim={dim} p={p} m={m} s={s}")
        self.dim, self.p, self.m = dim, p, m
        self.s = s if s > 0 else block_size(p)
        self.sched, self.tile, self.coarse, self.aggressive = sched, tile, coarse, aggressive
        self.n = lib.or_n(self._h)
        self.nc = lib.or_nc(self._h)
        self.N = lib.or_ndofs(self._h)
        self.Nc = self.nc ** dim

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_free(h)
            self._h = None

    def residual(self, u, b) -> np.ndarray:
        u = _f64(u); b = _f64(b)
        d = np.empty(self.N)
        self._lib.or_residual(self._h, _d(u), _d(b), _d(d))
        return d

    def apply_A(self, u) -> np.ndarray:
        return -self.residual(u, np.zeros(self.N))

    def smooth(self, u, b) -> np.ndarray:
        u = _f64(u).copy(); b = _f64(b)
        self._lib.or_smooth(self._h, _d(b), _d(u))
        return u

    def restrict(self, d) -> np.ndarray:
        d = _f64(d)
        dc = np.empty(self.Nc)
        self._lib.or_restrict(self._h, _d(d), _d(dc))
        return dc

    def prolong_add(self, ec, u) -> np.ndarray:
        ec = _f64(ec); u = _f64(u).copy()
        self._lib.or_prolong_add(self._h, _d(ec), _d(u))
        return u

    def coarse_solve(self, dc) -> np.ndarray:
        dc = _f64(dc)
        ec = np.empty(self.Nc)
        self._lib.or_coarse_solve(self._h, _d(dc), _d(ec))
        return ec

    def cycle(self, u, b, adjoint: bool = False) -> np.ndarray:
        u = _f64(u).copy(); b = _f64(b)
        fn = self._lib.or_cycle_adjoint if adjoint else self._lib.or_cycle
        fn(self._h, _d(b), _d(u))
        return u

    def solve(self, b, u0, tol: float = 1e-8, maxc: int = 100, adjoint: bool = False):
        """Returns (u, cycles, relres, history, converged)."""
        b = _f64(b); u = _f64(u0).copy()
        hist = np.zeros(maxc)
        cyc = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        st = self._lib.or_solve(self._h, _d(b), tol, maxc, int(adjoint), _d(u),
                                ctypes.byref(cyc), ctypes.byref(rel), _d(hist))
        return u, cyc.value, rel.value, hist[: cyc.value].copy(), st == 0
