#!/usr/bin/env python3
"""Benchmark: DOF/s to a 1e-8 relative residual on the paper's square-domain workload.

Workload (one step): the two-level solver of Algorithm 1 (LATTICE-coloured
multiplicative Schwarz, aggressive 2h degree-1 second level with one V(1,1)
cycle) run to ||b - A u|| <= 1e-8 ||b - A u_0|| on the 2D Poisson problem with
1024 x 1024 elements for each of p = 2, 3, 4, 5 (block sides 3, 3, 3, 5), FP64.
Inputs are synthetic and seeded: f has i.i.d. uniform[-1,1] B-spline
coefficients, b = (M (x) M) f, u_0 is i.i.d. uniform[-1,1] (SplitMix64).

value  = sum_p N_p / step time, inputs resident in HBM, L2 flushed before every solve;
         each solve is one iga2l_solve(f) call (b = (M (x) M) f formed by the library).
e2e    = the same through the public API with host buffers: H2D of f and u_0,
         iga2l_solve(f), D2H of u, all inside the timed region.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
N > 1 runs as one process per GPU: under torchrun as launched, or, when started
without a torchrun environment, bench.py starts N ranks itself through
torch.distributed.run.  Every rank solves the same workload independently
(replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M_ELEM = 1024
DEGREES = (2, 3, 4, 5)
TOL = 1e-8
COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3)}
METRIC = "DOF/s to 1e-8 rel. residual, mixed vs FP64; Schwarz sweep % of roofline"
WORKLOAD = ("2D Poisson on the unit square, B-splines p=2,3,4,5 (C^{p-1}), 1024x1024 elements "
            "(~1.05M DOFs each), seeded uniform[-1,1] coefficients of f, LATTICE-coloured "
            "multiplicative Schwarz + aggressive 2h linear second level with V(1,1), FP64, to 1e-8")
L2_BYTES = 129 * 1024 * 1024
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
ORACLE_CYCLES = os.path.join(ROOT, "tests", "golden", "oracle_cycles_m1024.json")
# FP64 pipe of GB300: 2 FP64 FMA per clock per SM, 152 SMs, 2070 MHz maximum SM clock
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070
# FP32 pipe of GB300: 128 FP32 FMA per clock per SM
FP32_PEAK_GFLOPS = 128 * 2 * 152 * 2.070


def seeds(p):
    from paper_2009_01499_gb300 import synth
    base = synth.BASE_SEED + 1
    return base + p, base + 10 + p


def schwarz_flops_per_dof(p, s, dim=2):
    """Algorithmic FP64 flops of one Schwarz block (one per DOF) as the FP64 colour kernel
    computes it: the block residual, the block solve with the precomputed inverse
    (s^{2d} multiply-adds) and the update (s^d adds).  3x3 and 5x5 blocks
    (k_schwarz_lattice2d): the residual as s^d rows of (2p+1)^d multiply-adds and one
    subtraction.  7x7 blocks in 2D (k_schwarz_lattice2d_pd, sum-factorised): s (s + 2p)
    pairs of (2p+1) multiply-adds (y pass), s^2 pairs of (2p+1) multiply-adds, one add
    and one subtraction (x pass)."""
    sd = s ** dim
    w = 2 * p + 1
    if dim == 2 and s >= 7:
        return 4 * w * s * (s + 2 * p) + 4 * w * sd + 2 * sd + 2 * sd * sd + sd
    return 2 * sd * w ** dim + sd + 2 * sd * sd + sd


def kernel_source_digest(relpath, function):
    """Hash of one kernel's definition text (from its name at the start of a line to the
    closing brace at the start of a line): a traffic record stays valid while that text
    is unchanged."""
    try:
        text = open(os.path.join(ROOT, relpath)).read()
    except OSError:
        return None
    start = text.find("\n" + function + "(")
    if start < 0:
        return None
    end = text.find("\n}\n", start)
    return hashlib.sha256(text[start:end].encode()).hexdigest()[:16] if end > 0 else None


def schwarz_flops_per_dof_f32(p, s):
    """Algorithmic FP32 flops of one Schwarz block (one per DOF) in the sum-factorised form of
    the FP32 kernels: y pass 2W s (s + 2p) and x pass 2W s^2 multiply-adds (pairs K, M), the
    block solve s^4 multiply-adds, one subtraction and one update per block DOF."""
    w = 2 * p + 1
    return 2 * (2 * w * s * (s + 2 * p) + 2 * w * s * s + s ** 4) + 2 * s * s


def block_side(p):
    return 3 if p <= 4 else 5


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- dist
def dist_setup(backend):
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, local, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, ws, device=None):
    """Maximum of a per-rank scalar over all ranks (the step time the job is charged)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- oracle
def host_cpu():
    """Core count and model of the host CPU (for the CPU-baseline lines)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_cycle_sample(degrees, cycles_per_p, threads=1):
    """Times one full-size oracle cycle plus one stopping-rule residual per degree and
    scales by the cycle counts: seconds the oracle needs to reach 1e-8 (threads > 1: the
    oracle's OpenMP build, identical results)."""
    import oracle
    from paper_2009_01499_gb300 import synth
    total = 0.0
    per = {}
    for p in degrees:
        q, g = COLOURING[p]
        O = oracle.Problem(2, p, M_ELEM, sched=oracle.LATTICE, coarse=oracle.VCYCLE, period=q, stride=g,
                           threads=threads)
        sf, su = seeds(p)
        f = synth.coefficients(O.N, sf)
        u0 = synth.initial_guess(O.N, su)
        _, Mm = oracle.assemble_1d(p, M_ELEM)
        b = (Mm @ f.reshape(O.n, O.n) @ Mm.T).ravel()
        t0 = time.perf_counter()
        d = O.residual(u0, b)
        np.linalg.norm(d)
        t1 = time.perf_counter()
        O.cycle(u0, b)
        t2 = time.perf_counter()
        t_res, t_cyc = t1 - t0, t2 - t1
        est = t_res + cycles_per_p[p] * (t_cyc + t_res)
        per[p] = {"cycle_s": t_cyc, "residual_s": t_res, "cycles": cycles_per_p[p], "solve_s_est": est}
        total += est
    return total, per


def oracle_full_solve(degrees, threads):
    """Times the oracle's whole solve to 1e-8 per degree (threads > 1: its OpenMP build,
    identical results): seconds and cycles per degree."""
    import oracle
    from paper_2009_01499_gb300 import synth
    total = 0.0
    per = {}
    for p in degrees:
        q, g = COLOURING[p]
        O = oracle.Problem(2, p, M_ELEM, sched=oracle.LATTICE, coarse=oracle.VCYCLE, period=q, stride=g,
                           threads=threads)
        sf, su = seeds(p)
        f = synth.coefficients(O.N, sf)
        u0 = synth.initial_guess(O.N, su)
        _, Mm = oracle.assemble_1d(p, M_ELEM)
        b = (Mm @ f.reshape(O.n, O.n) @ Mm.T).ravel()
        t0 = time.perf_counter()
        _, cyc, rel, _, ok = O.solve(b, u0, tol=TOL, maxc=100)
        dt = time.perf_counter() - t0
        per[p] = {"solve_s": dt, "cycles": int(cyc), "converged": bool(ok)}
        total += dt
    return total, per


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, same workload and metric."""
    if int(os.environ.get("RANK", "0")) != 0:
        return                      # under torchrun only rank 0 runs the reference
    import oracle
    from paper_2009_01499_gb300 import synth
    oracle.build()
    counts = {int(k): int(v) for k, v in json.load(open(ORACLE_CYCLES))["cycles"].items()}
    probs = {}
    ncores, model = host_cpu()
    for p in DEGREES:
        q, g = COLOURING[p]
        O = oracle.Problem(2, p, M_ELEM, sched=oracle.LATTICE, coarse=oracle.VCYCLE, period=q, stride=g,
                           threads=ncores)
        sf, su = seeds(p)
        f = synth.coefficients(O.N, sf)
        _, Mm = oracle.assemble_1d(p, M_ELEM)
        b = (Mm @ f.reshape(O.n, O.n) @ Mm.T).ravel()
        probs[p] = (O, b, synth.initial_guess(O.N, su))
    t_cyc = {p: [] for p in DEGREES}
    t_res = {p: [] for p in DEGREES}
    step_s = []

    def sample(p):
        O, b, u0 = probs[p]
        t0 = time.perf_counter()
        u1 = O.cycle(u0, b)
        t1 = time.perf_counter()
        np.linalg.norm(O.residual(u1, b))
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1

    for k in range(args.warmup + args.steps):
        p = DEGREES[k % len(DEGREES)]
        tc, tr = sample(p)
        if k >= args.warmup:
            t_cyc[p].append(tc)
            t_res[p].append(tr)
            step_s.append(tc + tr)
    total = 0.0
    for p in DEGREES:
        if not t_cyc[p]:            # degree not reached by the timed steps: one extra sample
            tc, tr = sample(p)
            t_cyc[p].append(tc)
            t_res[p].append(tr)
        tc, tr = statistics.mean(t_cyc[p]), statistics.mean(t_res[p])
        total += tr + counts[p] * (tc + tr)
    ndofs = sum(probs[p][0].N for p in DEGREES)
    value = ndofs / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(step_s),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "m": M_ELEM, "degrees": list(DEGREES),
                                        "tol": TOL, "dofs_per_step": ndofs},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": ncores, "kind": "oracle", "cpu": model,
                         "sample": f"oracle OpenMP build on {ncores} threads (bit-identical to one thread); "
                                   "each step: one full-size oracle cycle + stopping residual of one "
                                   "degree (p rotating 2,3,4,5); DOF/s = sum N_p / sum_p (t_res + "
                                   "cycles_p (t_cycle + t_res)), cycles_p = the oracle's own counts "
                                   "(tests/golden/oracle_cycles_m1024.json)"},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)



def _time_solve(S, f, u0, u, tol, stream, flush):
    flush.fill_(1.0)
    u.copy_(u0)
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    c, rel, _, ok = S.solve(f, u, tol=tol)
    e1.record(stream)
    e1.synchronize()
    if not ok:
        raise RuntimeError("solve did not converge")
    return e0.elapsed_time(e1), c


def concurrent_step(solvers, fs, us, u0s, flush, stream, streams, tol):
    """The four independent solves of one step at once: each on its own CUDA stream,
    driven by its own host thread (the library's calls release the GIL), L2 flushed
    once before the step.  Returns (ms, cycles per degree)."""
    import threading
    import torch
    flush.fill_(1.0)
    for p in solvers:
        us[p].copy_(u0s[p])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out, errors = {}, []

    def run(p):
        try:
            s = streams[p]
            s.wait_event(e0)
            c, rel, _, ok = solvers[p].solve(fs[p], us[p], tol=tol, stream=s)
            if not ok:
                raise RuntimeError(f"p={p} did not converge (rel {rel:.3e})")
            out[p] = c
        except Exception as exc:   # re-raised after the join
            errors.append(exc)

    threads = [threading.Thread(target=run, args=(p,)) for p in solvers]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for p in solvers:
        stream.wait_stream(streams[p])
    e1.record(stream)
    e1.synchronize()
    if errors:
        raise errors[0]
    return e0.elapsed_time(e1), out


def bench_3d(args, dev):
    """3D Poisson, p = 3 on 128^3 elements (2.15M DOFs), FP64 and mixed, to 1e-8."""
    import torch
    from paper_2009_01499_gb300 import iga2l, synth
    p, m = 3, 128
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    out = {"workload": "3D Poisson on the unit cube, p=3 on 128^3 elements (2,146,689 DOFs), seeded "
                       "uniform[-1,1] coefficients of f, LATTICE (7,2) colouring, 3x3x3 blocks, to 1e-8"}
    for name, prec in (("fp64", iga2l.FP64), ("mixed", iga2l.MIXED_FP32),
                       ("mixed_fp32_boundary", iga2l.MIXED_FP32_ALL)):
        S = iga2l.Solver(p, m, dim=3, period=7, stride=2, precision=prec)
        f = torch.tensor(synth.coefficients(S.N, synth.BASE_SEED + 3), device=dev)
        u0 = torch.tensor(synth.initial_guess(S.N, synth.BASE_SEED + 4), device=dev)
        u = torch.empty_like(u0)
        _time_solve(S, f, u0, u, TOL, stream, flush)
        runs = [_time_solve(S, f, u0, u, TOL, stream, flush) for _ in range(2)]
        ms = min(r[0] for r in runs)
        out[name] = {"value": S.N / (ms * 1e-3), "unit": "DOF/s", "ms": ms, "cycles": runs[-1][1]}
        S.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["speedup_mixed_fp32_boundary_vs_fp64"] = out["fp64"]["ms"] / out["mixed_fp32_boundary"]["ms"]
    return out


def bench_differentiable(args, dev):
    """p = 3 on 512^2 elements, f = 16 seeded Gaussian bumps (width 0.05), loss
    0.5 ||u - u_t||^2: forward solve + gradient w.r.t. the 48 bump parameters, by the adjoint
    solve (both solves to 1e-12) and by the unrolled 20-cycle backward; device time of one
    forward + backward each (CUDA events), and a central difference of the 40-cycle map for
    one parameter beside the adjoint gradient."""
    import torch
    from paper_2009_01499_gb300 import iga2l, synth
    from paper_2009_01499_gb300.autograd import bump_solve
    p, m, nb, width = 3, 512, 16, 0.05
    S = iga2l.Solver(p, m, period=7, stride=2)
    theta0 = synth.bumps(nb, synth.BASE_SEED + 5).ravel()
    ut = torch.tensor(synth.uniform_pm1(synth.BASE_SEED + 6, S.N), device=dev)

    def loss(th, mode, ncycles=20, tol=1e-12):
        u = bump_solve(th, S, width, mode=mode, tol=tol, ncycles=ncycles)
        return 0.5 * torch.sum((u - ut) ** 2)

    out = {"workload": "2D Poisson, p=3 on 512x512 elements, f = 16 seeded Gaussian bumps (width 0.05), loss "
                       "0.5||u - u_t||^2 with seeded u_t; gradient w.r.t. the 48 bump parameters"}
    grads = {}
    for mode in ("adjoint", "unrolled"):
        times = []
        for _ in range(3):
            th = torch.tensor(theta0, device=dev, requires_grad=True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            L = loss(th, mode)
            L.backward()
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            grads[mode] = th.grad.detach().cpu().numpy()
        out[mode] = {"ms_forward_backward": min(times[1:]), "loss": float(L.item())}
    idx = 0
    h = 1e-5 * max(1.0, abs(theta0[idx]))
    tp, tm = theta0.copy(), theta0.copy()
    tp[idx] += h
    tm[idx] -= h
    with torch.no_grad():
        fd = (loss(torch.tensor(tp, device=dev), "unrolled", ncycles=40).item()
              - loss(torch.tensor(tm, device=dev), "unrolled", ncycles=40).item()) / (2 * h)
    out["adjoint"]["fd_check"] = {"parameter": idx, "gradient": float(grads["adjoint"][idx]), "central_difference": fd,
                                  "rel_diff": float(abs(grads["adjoint"][idx] - fd) / max(1.0, abs(fd)))}
    g_a, g_u = grads["adjoint"], grads["unrolled"]
    out["unrolled"]["rel_diff_to_adjoint"] = float(np.abs(g_u - g_a).max() / np.abs(g_a).max())
    S.close()
    return out


def bench_high_degree(args, dev):
    """2D, p = 6, 7, 8 on 1024^2 elements (5x5 and 7x7 Schwarz blocks, Sections 4.3, 5.1):
    FP64 (LATTICE) and mixed (TILE for p = 6, LATTICE for 7x7 blocks), to 1e-8."""
    import torch
    from paper_2009_01499_gb300 import iga2l, synth
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    out = {"workload": "2D Poisson, B-splines p=6,7,8 on 1024x1024 elements, seeded uniform[-1,1] coefficients "
                       "of f, 5x5 (p=6) / 7x7 (p=7,8) blocks, colourings (11,4), (14,5), (17,4), to 1e-8"}
    for p in (6, 7, 8):
        row = {}
        for name, prec, sched in (("fp64", iga2l.FP64, iga2l.SCHED_LATTICE),
                                  ("mixed", iga2l.MIXED_FP32, iga2l.SCHED_TILE if p <= 6 else iga2l.SCHED_LATTICE)):
            S = iga2l.Solver(p, M_ELEM, precision=prec, schedule=sched)
            f = torch.tensor(synth.coefficients(S.N, synth.BASE_SEED + 10 + p), device=dev)
            u0 = torch.tensor(synth.initial_guess(S.N, synth.BASE_SEED + 20 + p), device=dev)
            u = torch.empty_like(u0)
            _time_solve(S, f, u0, u, TOL, stream, flush)
            runs = [_time_solve(S, f, u0, u, TOL, stream, flush) for _ in range(2)]
            ms = min(r[0] for r in runs)
            row[name] = {"value": S.N / (ms * 1e-3), "unit": "DOF/s", "ms": ms, "cycles": runs[-1][1],
                         "schedule": "TILE" if sched == iga2l.SCHED_TILE else "LATTICE"}
            S.close()
        row["speedup_mixed_vs_fp64"] = row["fp64"]["ms"] / row["mixed"]["ms"]
        out[str(p)] = row
    return out


def bench_batched(args, dev):
    """256 independent 2D problems, m from {64,128,256,512} and p from {2,3,4} by seed, solved
    to 1e-8 in the mixed form and in FP64, each with autotuned schedules and concurrent
    groups; device time between two events on the launching stream (the groups' streams
    wait on the first and are joined before the second)."""
    import numpy as np
    import torch
    from paper_2009_01499_gb300 import iga2l, synth
    from paper_2009_01499_gb300.batch import BatchedSolver
    nprob = 256
    z = synth.splitmix64(synth.BASE_SEED + 4, 2 * nprob)
    ms_choice = np.array([64, 128, 256, 512])[(z[0::2] % np.uint64(4)).astype(int)]
    ps = np.array([2, 3, 4])[(z[1::2] % np.uint64(3)).astype(int)]
    problems = [(int(p), int(m)) for p, m in zip(ps, ms_choice)]
    f = [torch.tensor(synth.coefficients((m + p - 2) ** 2, 1000 + i), device=dev) for i, (p, m) in enumerate(problems)]
    u0 = [torch.tensor(synth.initial_guess((m + p - 2) ** 2, 2000 + i), device=dev) for i, (p, m) in enumerate(problems)]
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "256 independent 2D Poisson problems, m uniform in {64,128,256,512}, p uniform in "
                       "{2,3,4} (seeded), uniform[-1,1] coefficients of f, to 1e-8",
           "timing": "CUDA events on the launching stream around the whole batch (groups on concurrent streams)"}
    for name, prec in (("mixed", iga2l.MIXED_FP32), ("fp64", iga2l.FP64)):
        BS = BatchedSolver(problems, precision=prec, autotune=True)
        fp = BS.pack(f)
        u0p = BS.pack(u0)
        ndofs = sum(BS.dofs)
        times, cycles = [], None
        for it in range(3):
            u = [t.clone() for t in u0p]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cycles, relres, ok = BS.solve(fp, u, tol=TOL)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            if not ok:
                raise RuntimeError(f"batched {name} solve did not converge")
        ms = min(times[1:])
        out[name] = {"value": ndofs / (ms * 1e-3), "unit": "DOF/s", "dofs": ndofs, "ms": ms,
                     "groups": len(BS.groups), "cycles_max": int(max(cycles)), "cycles": [int(c) for c in cycles],
                     "schedules": {f"p{g['p']}m{g['m']}": ("TILE" + (f"x{g['tile_groups']}" if g["tile_groups"] > 1
                                                                     else "")
                                                            + (" work-list" if g["sweep"] == iga2l.SWEEP_WORK_LIST
                                                               else "") if g["schedule"] == 2 else "LATTICE")
                                   for g in BS.groups}}
        BS.close()
    out["value"] = out["mixed"]["value"]
    out["unit"] = "DOF/s"
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms"] / out["mixed"]["ms"]
    out["cycles_equal"] = out["mixed"]["cycles"] == out["fp64"]["cycles"]
    for name in ("mixed", "fp64"):
        out[name].pop("cycles")
    return out

# ---------------------------------------------------------------------------- gpu arm
def run_gpu(args):
    import torch

    rank, local, ws = dist_setup("nccl")
    if ws != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but the world size is {ws}")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2009_01499_gb300 import iga2l, synth

    iga2l.load()
    solvers, fs, bs, u0s, us, fhost, u0host, uhost = {}, {}, {}, {}, {}, {}, {}, {}
    setup_ms = {}
    for p in DEGREES:
        q, g = COLOURING[p]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = iga2l.Solver(p, M_ELEM, period=q, stride=g)   # assemble: host tables + one upload
        torch.cuda.synchronize()
        setup_ms[str(p)] = round((time.perf_counter() - t0) * 1e3, 2)
        sf, su = seeds(p)
        f = torch.tensor(synth.coefficients(S.N, sf), device=dev)
        b = torch.empty_like(f)
        S.rhs_from_coeffs(f, b)      # b only for the sweep timing below; solves take f
        solvers[p], fs[p], bs[p] = S, f, b
        u0s[p] = torch.tensor(synth.initial_guess(S.N, su), device=dev)
        us[p] = torch.empty_like(u0s[p])
        fhost[p] = torch.tensor(synth.coefficients(S.N, sf)).pin_memory()
        u0host[p] = torch.tensor(synth.initial_guess(S.N, su)).pin_memory()
        uhost[p] = torch.empty(S.N, dtype=torch.float64).pin_memory()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ndofs = sum(solvers[p].N for p in DEGREES)

    def step(timed):
        tot_ms, cyc = 0.0, {}
        for p in DEGREES:
            flush.fill_(1.0)                       # evict L2 before every solve
            us[p].copy_(u0s[p])
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c, rel, _, ok = solvers[p].solve(fs[p], us[p], tol=TOL)
            e1.record(stream)
            e1.synchronize()
            if not ok:
                raise RuntimeError(f"p={p} did not converge (rel {rel:.3e})")
            tot_ms += e0.elapsed_time(e1)
            cyc[p] = c
        return tot_ms, cyc

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    barrier(ws)
    l0 = iga2l.kernel_launches()
    step_ms, cycles = [], None
    for _ in range(args.steps):
        ms, cycles = step(True)
        step_ms.append(ms)
    launches = iga2l.kernel_launches() - l0
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ms_step = allmax(statistics.mean(step_ms), ws, dev)
    value = ws * ndofs / (ms_step * 1e-3)

    # the same step with the four solves running concurrently (one stream and host thread each)
    cstreams = {p: torch.cuda.Stream(dev) for p in DEGREES}
    for _ in range(args.warmup):
        concurrent_step(solvers, fs, us, u0s, flush, stream, cstreams, TOL)
    cms = [concurrent_step(solvers, fs, us, u0s, flush, stream, cstreams, TOL)[0] for _ in range(args.steps)]
    c_ms = allmax(statistics.mean(cms), ws, dev)
    concurrent = {"value": ws * ndofs / (c_ms * 1e-3), "unit": "DOF/s", "ms_per_step": c_ms,
                  "note": "the step's four independent solves on four streams at once (L2 flushed once per step)"}

    # end to end through the public API with host buffers (H2D, rhs, solve, D2H)
    h2d = d2h = 0
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        tot = 0.0
        for p in DEGREES:
            S = solvers[p]
            flush.fill_(1.0)
            f_dev = torch.empty(S.N, dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f_dev.copy_(fhost[p], non_blocking=True)
            us[p].copy_(u0host[p], non_blocking=True)
            S.solve(f_dev, us[p], tol=TOL)
            uhost[p].copy_(us[p], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
            if it == 0:
                h2d += fhost[p].numel() * 8 + u0host[p].numel() * 8
                d2h += uhost[p].numel() * 8
        if it >= args.warmup:
            e2e_ms.append(tot)
    e2e_step = allmax(statistics.mean(e2e_ms), ws, dev)

    # mixed precision (FP32 inner cycle, TILE schedule) inside FP64 refinement, same
    # workload and stopping rule: boundary-block inverses applied in FP64 ("mixed") or
    # in FP32 as well ("mixed_fp32_boundary")
    mixed, mixed_all, mixed_tf32, mixed_same = None, None, None, None
    # FMA-pipe throughputs of this GPU, measured now (the ALU rooflines' denominators)
    peaks = {"fp64": iga2l.fma_peak(0), "fp32": iga2l.fma_peak(1), "fp32x2": iga2l.fma_peak(2)}
    if not args.no_mixed:

        def run_mixed(precision, boundary, schedules):
            msolv = {}
            for p in DEGREES:
                q, g = COLOURING[p]
                msolv[p] = iga2l.Solver(p, M_ELEM, period=q, stride=g, precision=precision, schedule=schedules[p])
            mcyc = {}

            def mstep():
                tot = 0.0
                for p in DEGREES:
                    flush.fill_(1.0)
                    us[p].copy_(u0s[p])
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    c, rel, _, ok = msolv[p].solve(fs[p], us[p], tol=TOL)
                    e1.record(stream)
                    e1.synchronize()
                    if not ok:
                        raise RuntimeError(f"mixed p={p} did not converge")
                    tot += e0.elapsed_time(e1)
                    mcyc[p] = c
                return tot

            for _ in range(args.warmup):
                mstep()
            mms = allmax(statistics.mean([mstep() for _ in range(args.steps)]), ws, dev)
            for _ in range(args.warmup):
                concurrent_step(msolv, fs, us, u0s, flush, stream, cstreams, TOL)
            mcms = allmax(statistics.mean([concurrent_step(msolv, fs, us, u0s, flush, stream, cstreams, TOL)[0]
                                           for _ in range(args.steps)]), ws, dev)

            def sched_name(S):
                if S.tile:
                    return f"TILE({S.tile})" + (f"x{S.tile_groups} groups" if S.tile_groups > 1 else "")
                return "LATTICE"

            out = {"value": ws * ndofs / (mms * 1e-3), "unit": "DOF/s", "ms_per_step": mms,
                   "speedup_vs_fp64": ms_step / mms,
                   "dtype": f"f32 inner cycle ({boundary} boundary-block inverses), f64 residual/update/coarsest",
                   "schedule": {str(p): sched_name(msolv[p]) for p in DEGREES},
                   "cycles": {str(p): mcyc[p] for p in DEGREES},
                   "cycles_equal_fp64": all(mcyc[p] == cycles[p] for p in DEGREES),
                   "accuracy": "same 1e-8 FP64 residual rule; refined to 1e-12 the solution is within "
                               "1e-8 of the FP64 oracle's (tests/test_gpu_mixed.py)",
                   "concurrent": {"value": ws * ndofs / (mcms * 1e-3), "unit": "DOF/s", "ms_per_step": mcms}}
            return out, msolv

        def sweep_roofline(msolv):
            """FP32 Schwarz sweep of the inner cycle (iga2l_schwarz_sweep_f32), timed alone with
            CUDA events on the FP32 copies of the step's vectors (L2-resident, as inside a solve)."""
            tot_fl, tot_ms, per = 0.0, 0.0, {}
            for p in DEGREES:
                S = msolv[p]
                u32 = u0s[p].float()
                b32 = bs[p].float()
                S.schwarz_sweep_f32(u32, b32)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 5
                e0.record(stream)
                for _ in range(reps):
                    S.schwarz_sweep_f32(u32, b32)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / reps
                fl = schwarz_flops_per_dof_f32(p, block_side(p)) * S.N
                per[str(p)] = {"sweep_ms": round(ms, 4), "gflops": round(fl / ms / 1e6, 1),
                               "cycles": msolv_cycles[p], "schedule": sched_of[str(p)]}
                tot_fl += msolv_cycles[p] * fl
                tot_ms += msolv_cycles[p] * ms
            ach = tot_fl / tot_ms / 1e6
            pk = FP32_PEAK_GFLOPS
            return {"bound": "alu", "achieved": round(ach, 1), "peak": round(pk, 1), "unit": "GFLOP/s",
                    "frac": round(ach / pk, 4), "traffic": None,
                    "kernel": "FP32 Schwarz sweep of the inner cycle (TILE: k_schwarz_tile2d; LATTICE: one launch per "
                              "colour or k_schwarz_persist2d)",
                    "peak_source": "FP32 FMA pipe from unit counts: 128 FMA/clk/SM x 152 SMs x 2070 MHz (the "
                                   "packed pair instruction issues two of them); dependent-free FMA loops measured "
                                   f"{peaks['fp32']:.0f} (scalar) and {peaks['fp32x2']:.0f} (pairs) GFLOP/s in this "
                                   "run (iga2l_fma_peak)",
                    "flops": "sum-factorised block residual + block solve per DOF: 2[2W s(s+2p) + 2W s^2 + s^4] "
                             "+ 2 s^2, W = 2p+1",
                    "per_degree": per}

        # headline mixed form: per degree the fastest schedule with the FP64 form's cycle counts
        best = {2: iga2l.SCHED_TILE, 3: iga2l.SCHED_TILE, 4: iga2l.SCHED_LATTICE, 5: iga2l.SCHED_TILE}
        mixed, msolv = run_mixed(iga2l.MIXED_FP32, "f64", best)
        msolv_cycles = {p: mixed["cycles"][str(p)] for p in DEGREES}
        sched_of = mixed["schedule"]
        mixed["roofline"] = sweep_roofline(msolv)
        for S in msolv.values():
            S.close()
        mixed_all, ms_ = run_mixed(iga2l.MIXED_FP32_ALL, "f32", best)
        for S in ms_.values():
            S.close()
        # the same schedule as the FP64 form (LATTICE for every degree)
        mixed_same, ms_ = run_mixed(iga2l.MIXED_FP32, "f64", {p: iga2l.SCHED_LATTICE for p in DEGREES})
        for S in ms_.values():
            S.close()
        # the interior blocks of every LATTICE colour as a tcgen05 TF32 GEMM
        mixed_tf32, ms_ = run_mixed(iga2l.MIXED_TF32, "f64", {p: iga2l.SCHED_LATTICE for p in DEGREES})
        for S in ms_.values():
            S.close()
        mixed_tf32["dtype"] = ("tf32 tensor-core interior block solves (tcgen05, f32 accumulation), f32 boundary "
                               "frame, f64 residual/update/coarsest")

    # secondary configurations: 3D (p = 3, 128^3, FP64 and mixed), the batch of 256 uneven
    # 2D problems (mixed, autotuned schedules, concurrent groups), and p = 6..8 at 1024^2
    extra = {}
    if not args.no_extra:
        extra["3d"] = bench_3d(args, dev)
        extra["batched"] = bench_batched(args, dev)
        extra["high_degree"] = bench_high_degree(args, dev)
        extra["differentiable"] = bench_differentiable(args, dev)

    # roofline of the dominant kernel, the Schwarz colour-phase kernel (FP64 pipe bound)
    sweep_flops, sweep_ms, per_p = 0.0, 0.0, {}
    for p in DEGREES:
        S = solvers[p]
        u = us[p]
        u.copy_(u0s[p])
        S.schwarz_sweep(u, bs[p])
        reps = 3
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            S.schwarz_sweep(u, bs[p])
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        q = COLOURING[p][0]
        fl = schwarz_flops_per_dof(p, block_side(p)) * S.N
        per_p[str(p)] = {"sweep_ms": round(ms, 4), "launches_per_sweep": q * q,
                         "gflops": round(fl / ms / 1e6, 1), "cycles": cycles[p]}
        sweep_flops += cycles[p] * fl
        sweep_ms += cycles[p] * ms
    achieved = sweep_flops / sweep_ms / 1e6   # GFLOP/s
    traffic = None
    if os.path.exists(TRAFFIC_FILE):
        rec = json.load(open(TRAFFIC_FILE))
        if rec.get("kernel_source_sha256_16") == kernel_source_digest(rec.get("source", ""), rec.get("function", "")):
            traffic = rec.get("bytes_per_launch")
    roofline = {"bound": "alu", "achieved": round(achieved, 1), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4), "traffic": traffic,
                "kernel": "k_schwarz_lattice2d (one colour phase per launch)",
                "peak_source": "FP64 FMA pipe from unit counts: 2 FMA/clk/SM x 152 SMs x 2070 MHz (ncu reports "
                               "the same 2 FP64 FMA per SM and cycle); a dependent-free FMA loop measured "
                               f"{peaks['fp64']:.1f} GFLOP/s in this run (iga2l_fma_peak)",
                "per_degree": per_p}

    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M_ELEM, "degrees": list(DEGREES), "tol": TOL,
                   "dofs_per_step": ndofs, "cycles": {str(p): cycles[p] for p in DEGREES},
                   "l2": "flushed (256 MiB write) before every solve", "schedule": "LATTICE",
                   "setup_ms": setup_ms,
                   "colouring": {str(p): list(COLOURING[p]) for p in DEGREES},
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": ws * ndofs / (e2e_step * 1e-3), "unit": "DOF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "clocks": clk,
        "concurrent": concurrent, "mixed": mixed, "mixed_fp32_boundary": mixed_all,
        "mixed_same_schedule_as_fp64": mixed_same, "mixed_tf32_tensor_core": mixed_tf32,
        "measured_peaks_gflops": peaks or None,
        "other_configs": extra,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ncores, model = host_cpu()
        counts = {p: cycles[p] for p in DEGREES}
        total_n, per_n = oracle_full_solve(DEGREES, threads=ncores)
        total_1, per_1 = oracle_cycle_sample(DEGREES, counts, threads=1)
        line["cpu_baseline"] = {
            "value": ndofs / total_n, "unit": "DOF/s", "cores": ncores, "kind": "oracle",
            "cpu": model,
            "sample": f"the oracle's OpenMP build on {ncores} threads (blocks of a colour, sub-lattice points, "
                      "stencil and transfer outputs in parallel; results bit-identical to one thread): the whole "
                      "solve to 1e-8 of each degree's problem, timed: "
                      + ", ".join(f"p={p}: {v['solve_s']:.2f}s, {v['cycles']} cycles" for p, v in per_n.items()),
            "cycles_equal_gpu": all(per_n[p]["cycles"] == cycles[p] for p in DEGREES),
            "single_thread": {"value": ndofs / total_1, "unit": "DOF/s", "cores": 1,
                              "estimate": "one full-size cycle + one stopping residual per degree on one thread, "
                                          "scaled by the cycle counts (a whole one-thread solve takes about a "
                                          "minute)",
                              "per_degree_cycle_s": {str(p): round(v["cycle_s"], 3) for p, v in per_1.items()}}}
    elif rank == 0:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_profile_step(args):
    """For ncu: --warmup solves per degree, then one solve per degree, nothing else.  The
    solvers use plain launches (graphs off): ncu does not list the kernels that run inside
    a graph's conditional WHILE node (the device-driven solve), and per-kernel durations
    and counters do not depend on how the kernels were launched."""
    import torch
    from paper_2009_01499_gb300 import iga2l, synth
    dev = torch.device("cuda", 0)
    dim = args.profile_dim
    degrees = (args.profile_p,) if args.profile_p else ((3,) if dim == 3 else DEGREES)
    m = args.profile_m or (128 if dim == 3 else M_ELEM)
    prec = {"fp64": iga2l.FP64, "mixed": iga2l.MIXED_FP32, "mixed_all": iga2l.MIXED_FP32_ALL,
            "mixed_tf32": iga2l.MIXED_TF32}[args.profile_precision]
    best = {2: iga2l.SCHED_TILE, 3: iga2l.SCHED_TILE, 4: iga2l.SCHED_LATTICE, 5: iga2l.SCHED_TILE}
    if args.profile_schedule == "best":     # the benchmark's mixed schedules per degree
        sched = None
    elif args.profile_schedule:
        sched = iga2l.SCHED_TILE if args.profile_schedule == "tile" else iga2l.SCHED_LATTICE
    else:
        sched = iga2l.SCHED_LATTICE if (prec in (iga2l.FP64, iga2l.MIXED_TF32) or dim == 3) else iga2l.SCHED_TILE
    sweep = {"auto": iga2l.SWEEP_AUTO, "per_colour": iga2l.SWEEP_PER_COLOUR,
             "persistent": iga2l.SWEEP_PERSISTENT}[args.profile_sweep]
    for p in degrees:
        col = {"period": COLOURING[p][0], "stride": COLOURING[p][1]} if p in COLOURING else {}   # else the default
        sch = sched if sched is not None else best.get(p, iga2l.SCHED_LATTICE)
        S = iga2l.Solver(p, m, dim=dim, precision=prec, schedule=sch, graphs=0, sweep=sweep, **col)
        sf, su = seeds(p)
        f = torch.tensor(synth.coefficients(S.N, sf), device=dev)
        u0 = torch.tensor(synth.initial_guess(S.N, su), device=dev)
        u = torch.empty_like(u0)
        for _ in range(args.warmup + 1):
            u.copy_(u0)
            cyc, rel, _, ok = S.solve(f, u, tol=TOL)
        torch.cuda.synchronize()
        print(f"p={p} m={m} dim={dim}: {cyc} cycles, rel {rel:.3e}, converged {ok}", flush=True)
        S.close()


def _free_port():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def relaunch_as_ranks(args, argv):
    """--gpus N > 1 without a torchrun environment: start N ranks (one process per GPU)
    through torch.distributed.run on this node and return its exit status."""
    if not args.launch_check and args.impl == "gpu":
        import torch
        have = torch.cuda.device_count() if torch.cuda.is_available() else 0
        if have < args.gpus:
            raise SystemExit(f"bench.py: --gpus {args.gpus} requested but only {have} GPU(s) are visible")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(args.gpus),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.abspath(__file__)] + argv
    return subprocess.call(cmd)


def run_launch_check(args):
    """Launcher check without GPU work: every rank joins the process group (gloo without
    CUDA), reports a per-rank time, and rank 0 prints the job line with the world size."""
    backend = "nccl" if args.impl == "gpu" and _cuda_ok() else "gloo"
    rank, local, ws = dist_setup(backend)
    if ws != args.gpus:
        raise SystemExit(f"bench.py: --gpus {args.gpus} but the world size is {ws}")
    barrier(ws)
    ms = allmax(1.0 + rank, ws)
    if rank == 0:
        print(json.dumps({"launch_check": True, "n_gpus": ws, "ms_per_step": ms, "backend": backend}), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _cuda_ok():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the 3D and batched configurations")
    ap.add_argument("--profile-step", action="store_true",
                    help="profiling aid: warm-up solves then one solve per degree, no timing")
    ap.add_argument("--profile-m", type=int, default=0, help="elements per axis (default 1024 in 2D, 128 in 3D)")
    ap.add_argument("--profile-dim", type=int, choices=[2, 3], default=2)
    ap.add_argument("--profile-p", type=int, default=0)
    ap.add_argument("--profile-precision", choices=["fp64", "mixed", "mixed_all", "mixed_tf32"], default="fp64",
                    help="form profiled by --profile-step (the benchmark's schedule for it)")
    ap.add_argument("--profile-schedule", choices=["lattice", "tile", "best"], default=None,
                    help="schedule profiled by --profile-step (default: the benchmark's for the form)")
    ap.add_argument("--profile-sweep", choices=["auto", "per_colour", "persistent"], default="auto",
                    help="FP32 inner sweep kernel profiled by --profile-step")
    ap.add_argument("--launch-check", action="store_true",
                    help="start the ranks and report the world size, without GPU work (launcher test)")
    argv = sys.argv[1:]
    args = ap.parse_args(argv)
    if args.gpus < 1:
        ap.error("--gpus must be >= 1")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(relaunch_as_ranks(args, argv))
    if args.launch_check:
        run_launch_check(args)
        return
    if args.profile_step:
        run_profile_step(args)
        return
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
