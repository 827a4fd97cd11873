"""Batched solves of many independent 2D problems of uneven size and degree.

Problems are grouped by (p, m); each group is one batch handle of the library
(shared tables, one launch per step for the whole group, converged problems
masked on the device, cycles replayed from captured CUDA graphs).  Groups run
concurrently, each on its own CUDA stream driven by its own host thread (the
library's calls release the GIL).  For every group the schedule of the Schwarz step
(LATTICE, or TILE with its colours in 1, 2 or 4 groups, each TILE form either one launch
per tile phase or the work-list sweep: one launch per sweep over every problem's tiles)
is chosen by timing a seeded probe batch of the group's size to 1e-8 with each candidate,
so a candidate that costs cycles loses what it saves per cycle; choices are cached per
(device, p, m, precision, batch size), in memory and optionally in a JSON file.

This module is host orchestration only: all arithmetic runs in libiga2l.so.
"""
from __future__ import annotations

import json
import os
import threading
from collections import OrderedDict

import numpy as np
import torch

from . import iga2l, synth

COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3), 6: (11, 4), 7: (14, 5), 8: (17, 4)}
# (schedule, TILE colour groups, sweep form); TILE is compiled for blocks up to 5x5 (p <= 6)
CANDIDATES = tuple([(iga2l.SCHED_LATTICE, 0, iga2l.SWEEP_AUTO)] +
                   [(iga2l.SCHED_TILE, gr, sw) for sw in (iga2l.SWEEP_AUTO, iga2l.SWEEP_WORK_LIST) for gr in (1, 2, 4)])
_cache: dict = {}
_cache_lock = threading.Lock()


def _key(p, m, precision, nbatch):
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return f"{name}|p={p}|m={m}|prec={precision}|nbatch={nbatch}"


def autotune_schedule(p: int, m: int, precision: int, cache_path: str | None = None, reps: int = 2,
                      nbatch: int = 1):
    """Fastest (schedule, TILE colour groups, sweep form) by the time to a 1e-8 residual of a
    seeded probe batch of nbatch problems of the same (p, m) (one problem: a single-problem
    handle): the latency of small grids and the throughput of large batches pick differently."""
    key = _key(p, m, precision, nbatch)
    with _cache_lock:
        if key in _cache and len(_cache[key]) == 3:
            return _cache[key]
        if cache_path and os.path.exists(cache_path):
            try:
                _cache.update(json.load(open(cache_path)))
            except (OSError, ValueError):
                pass
            if key in _cache and len(_cache[key]) == 3:
                return _cache[key]
    q, g = COLOURING[p]
    best, best_ms = None, float("inf")
    for sched, groups, sweep in CANDIDATES:
        if sched == iga2l.SCHED_TILE and p > 6:   # TILE is compiled for blocks up to 5x5
            continue
        S = iga2l.Solver(p, m, period=q, stride=g, precision=precision, schedule=sched, tile_groups=groups,
                         sweep=sweep, nbatch=nbatch, batch=nbatch > 1)
        N = (m + p - 2) ** 2
        f = torch.tensor(np.concatenate([synth.coefficients(N, 77 + k) for k in range(nbatch)]), device="cuda")
        u0 = torch.tensor(np.concatenate([synth.initial_guess(N, 78 + k) for k in range(nbatch)]), device="cuda")
        times = []
        for _ in range(reps + 1):
            u = u0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            if nbatch > 1:
                S.solve_batch(f, u, tol=1e-8)
            else:
                S.solve(f, u, tol=1e-8)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = min(times[1:])
        S.close()
        if ms < best_ms:
            best, best_ms = [sched, groups, sweep], ms
    with _cache_lock:
        _cache[key] = best
        if cache_path:
            try:
                with open(cache_path, "w") as fh:
                    json.dump(_cache, fh, indent=1)
            except OSError:
                pass
    return best


class BatchedSolver:
    """Independent 2D problems given as a list of (p, m), solved group by group."""

    def __init__(self, problems, precision: int = iga2l.MIXED_FP32, autotune: bool = True,
                 cache_path: str | None = None, schedule: int | None = None, rhs_is_load: bool = False,
                 sweep: int = iga2l.SWEEP_AUTO):
        self.problems = list(problems)
        self.precision = precision
        groups: "OrderedDict[tuple, list]" = OrderedDict()
        for idx, (p, m) in enumerate(self.problems):
            groups.setdefault((p, m), []).append(idx)
        self.groups = []
        for (p, m), members in groups.items():
            if schedule is not None:
                sched, groups_, sweep_ = schedule, 0, sweep
            elif autotune:
                sched, groups_, sweep_ = autotune_schedule(p, m, precision, cache_path, nbatch=len(members))
            else:
                sched, groups_, sweep_ = iga2l.SCHED_LATTICE, 0, iga2l.SWEEP_AUTO
            q, g = COLOURING[p]
            h = iga2l.Solver(p, m, nbatch=len(members), batch=True, period=q, stride=g, precision=precision,
                             schedule=sched, tile_groups=groups_, sweep=sweep_,
                             rhs=iga2l.RHS_IS_LOAD if rhs_is_load else iga2l.RHS_COEFFS)
            self.groups.append({"p": p, "m": m, "members": members, "handle": h, "schedule": sched,
                                "tile_groups": h.tile_groups, "sweep": sweep_, "stream": torch.cuda.Stream()})
        self.dofs = [(m + p - 2) ** 2 for p, m in self.problems]

    def pack(self, vectors):
        """Per-problem vectors -> one packed device tensor per group."""
        return [torch.cat([vectors[i].reshape(-1) for i in g["members"]]).contiguous() for g in self.groups]

    def unpack(self, packed):
        out = [None] * len(self.problems)
        for g, t in zip(self.groups, packed):
            N = g["handle"].N
            for k, i in enumerate(g["members"]):
                out[i] = t[k * N:(k + 1) * N]
        return out

    def rhs_from_coeffs(self, f_packed):
        """b = (M x M) f for every problem (packed per group)."""
        b_packed = []
        for g, f in zip(self.groups, f_packed):
            b = torch.empty_like(f)
            with torch.cuda.stream(g["stream"]):
                g["handle"].rhs_from_coeffs(f, b, stream=g["stream"])
            b_packed.append(b)
        for g in self.groups:
            g["stream"].synchronize()
        return b_packed

    def solve(self, rhs_packed, u_packed, tol: float = 1e-8, max_cycles: int = 0):
        """Solves all groups concurrently in place; rhs_packed holds the coefficient vectors f
        of every problem (load vectors b with rhs_is_load=True).  Returns (cycles, relres,
        converged) per problem."""
        cycles = [0] * len(self.problems)
        relres = [0.0] * len(self.problems)
        ok = [True]
        errors = []

        def run(g, b, u):
            try:
                c, r, conv = g["handle"].solve_batch(b, u, tol=tol, max_cycles=max_cycles, stream=g["stream"])
                for k, i in enumerate(g["members"]):
                    cycles[i], relres[i] = int(c[k]), float(r[k])
                if not conv:
                    ok[0] = False
            except Exception as exc:   # reported after all threads join
                errors.append(exc)

        cur = torch.cuda.current_stream()
        for g in self.groups:
            g["stream"].wait_stream(cur)
        threads = [threading.Thread(target=run, args=(g, b, u)) for g, b, u in zip(self.groups, rhs_packed, u_packed)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for g in self.groups:
            cur.wait_stream(g["stream"])
        if errors:
            raise errors[0]
        return cycles, relres, ok[0]

    def close(self):
        for g in self.groups:
            g["handle"].close()
