"""Guard zones in place of a memory checker (GPU).

A handle assembled with IGA2L_TEST_GUARD_ALLOCS places every device buffer it allocates
between guard zones: NaN bytes around floating-point buffers, zero bytes around integer
tables and counters.  Here every vector handed to the library also sits inside a buffer
whose 4 KiB on either side hold NaNs.  A kernel that reads past the end of a floating-point
buffer therefore meets a NaN that reaches its results, and one that writes past either end
of any buffer changes a zone.

Every entry point of every form runs twice, on a guarded handle with guarded vectors and on
a plain handle with plain ones:
  * forms: FP64; the three mixed forms; LATTICE, TILE, work-list and persistent sweeps;
    2D and 3D; batches;
  * sizes: the smallest grids the parity tests use for each form, where boundary blocks
    and boundary stencil rows are much of the work, and for the 2D forms that accept them
    the smallest grids of all, where every block and every row is a boundary one.
The results must be finite and bitwise those of the plain run, the library's zones must be
unchanged (iga2l_guard_check) and the vectors' zones must still hold their NaNs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

G = 512   # guard words on each side of a vector handed to the library (4 KiB of float64)
COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3), 6: (11, 4), 7: (14, 5), 8: (17, 4)}


class Vectors:
    """Makes the vectors of one run: plain CUDA tensors, or views into NaN-guarded buffers."""

    def __init__(self, guarded):
        self.guarded = guarded
        self.buffers = []

    def __call__(self, host, dtype=torch.float64):
        host = torch.as_tensor(np.asarray(host), dtype=dtype)
        if not self.guarded:
            return host.to("cuda")
        buf = torch.full((host.numel() + 2 * G,), float("nan"), dtype=dtype, device="cuda")
        buf[G:G + host.numel()] = host.to("cuda")
        self.buffers.append((buf, buf[:G].clone()))
        return buf[G:G + host.numel()]

    def zones_intact(self):
        itype = {torch.float64: torch.int64, torch.float32: torch.int32}
        for buf, zone in self.buffers:
            it = itype[buf.dtype]
            for z in (buf[:G], buf[-G:]):
                if not torch.equal(z.view(it), zone.view(it)):
                    return False
        return True


def _exercise(S, mk, seed):
    """Every single-problem entry point of handle S once; returns the named results."""
    N, Nc = S.N, S.Nc
    f = mk(synth.coefficients(N, seed))
    u0 = synth.initial_guess(N, seed + 1)
    out = {}
    b = mk(np.zeros(N))
    S.rhs_from_coeffs(f, b)
    out["b"] = b
    y = mk(np.zeros(N))
    S.apply_A(mk(u0), y)
    out["Au"] = y
    d = mk(np.zeros(N))
    out["norm"] = torch.tensor([S.residual(mk(u0), b, d, want_norm=True)])
    out["d"] = d
    for rev in (False, True):
        u = mk(u0)
        S.schwarz_sweep(u, b, reverse=rev)
        out[f"sweep_rev{int(rev)}"] = u
    if S.options.precision != iga2l.FP64 and S.dim == 2:
        for rev in (False, True):
            uf = mk(u0, torch.float32)
            S.schwarz_sweep_f32(uf, mk(synth.coefficients(N, seed + 2), torch.float32), reverse=rev)
            out[f"sweep_f32_rev{int(rev)}"] = uf
    dc = mk(np.zeros(Nc))
    S.restrict(d, dc)
    out["dc"] = dc
    ec = mk(np.zeros(Nc))
    S.coarse_solve(dc, ec)
    out["ec"] = ec
    u = mk(u0)
    S.prolong_add(ec, u)
    out["prolong"] = u
    for adj in (False, True):
        u = mk(u0)
        S.cycle(u, b, adjoint=adj)
        out[f"cycle_adj{int(adj)}"] = u
    u = mk(u0)
    S.cycles(u, b, 2)
    out["cycles"] = u
    u = mk(u0)
    c, rel, _, _ = S.solve(f, u, tol=1e-8, max_cycles=40)
    out["solve"], out["solve_stats"] = u, torch.tensor([c, rel])
    u = mk(u0)
    c, rel, _, _ = S.solve_load(b, u, tol=1e-8, max_cycles=40)
    out["solve_load"], out["solve_load_stats"] = u, torch.tensor([c, rel])
    lam = mk(np.zeros(N))
    c, rel, _ = S.adjoint_solve(mk(synth.coefficients(N, seed + 3)), lam, tol=1e-8, max_cycles=40)
    out["adjoint"], out["adjoint_stats"] = lam, torch.tensor([c, rel])
    bbar = mk(np.zeros(N))
    S.unrolled_backward(mk(synth.coefficients(N, seed + 4)), 3, bbar)
    out["unrolled"] = bbar
    if S.dim == 2:
        theta = mk(synth.bumps(4, seed + 5).ravel())
        bl = mk(np.zeros(N))
        S.bump_load(theta, 0.05, bl)
        out["bump_load"] = bl
        grad = mk(np.zeros(12))
        S.bump_grad(theta, 0.05, mk(synth.coefficients(N, seed + 6)), grad)
        out["bump_grad"] = grad
    return out


def _compare(plain, guarded):
    assert plain.keys() == guarded.keys()
    for k in plain:
        a, g = plain[k].cpu(), guarded[k].cpu()
        assert torch.isfinite(g).all(), f"{k}: non-finite values (a read outside a buffer)"
        assert torch.equal(a, g), f"{k}: differs from the unguarded run"


def _run(make, seed, exercise=_exercise):
    results, handles, vecs = [], [], []
    for guarded in (False, True):
        S = make(guarded)
        mk = Vectors(guarded)
        results.append(exercise(S, mk, seed))
        torch.cuda.synchronize()
        handles.append(S)
        vecs.append(mk)
    _compare(*results)
    assert handles[1].guard_check() == 0, "a kernel wrote into a guard zone of the library's buffers"
    assert vecs[1].zones_intact(), "a kernel wrote outside a vector handed to it"


def _solver(p, m, guarded, **kw):
    if kw.get("dim", 2) == 2 and "period" not in kw:
        kw["period"], kw["stride"] = COLOURING[p]
    return iga2l.Solver(p, m, test_flags=iga2l.TEST_GUARD_ALLOCS if guarded else 0, **kw)


FP64_2D = [(2, 24, "lattice"), (3, 26, "lattice"), (4, 30, "lattice"), (5, 28, "lattice"),
           (6, 50, "lattice"), (7, 40, "lattice"), (8, 44, "lattice"),
           (2, 24, "tile"), (3, 26, "tile"), (4, 30, "tile"), (5, 28, "tile"), (6, 50, "tile"),
           (2, 12, "work_list"), (3, 16, "work_list"),
           # the smallest grids: every block and every stencil row a boundary one
           (2, 4, "lattice"), (3, 4, "lattice"), (4, 6, "lattice"), (5, 6, "lattice"), (6, 8, "lattice"),
           (7, 8, "lattice"), (8, 10, "lattice"), (2, 4, "tile"), (4, 6, "tile"), (5, 6, "tile"),
           (3, 4, "work_list"), (6, 8, "work_list")]


def _sched_kw(sched):
    if sched == "lattice":
        return {"schedule": iga2l.SCHED_LATTICE}
    if sched == "lattice_pc":
        return {"schedule": iga2l.SCHED_LATTICE, "sweep": iga2l.SWEEP_PER_COLOUR}
    if sched == "persistent":
        return {"schedule": iga2l.SCHED_LATTICE, "sweep": iga2l.SWEEP_PERSISTENT}
    if sched == "tile":
        return {"schedule": iga2l.SCHED_TILE}
    return {"schedule": iga2l.SCHED_TILE, "sweep": iga2l.SWEEP_WORK_LIST}


@pytest.mark.parametrize("p,m,sched", FP64_2D)
def test_fp64_2d_stays_inside_its_buffers(p, m, sched):
    _run(lambda gd: _solver(p, m, gd, **_sched_kw(sched)), 500 + p)


MIXED_2D = [(iga2l.MIXED_FP32, p, m, s) for (p, m) in [(2, 50), (3, 64), (4, 66), (5, 70)]
            for s in ("lattice_pc", "tile", "work_list")]
MIXED_2D += [(iga2l.MIXED_FP32, 2, 50, "persistent"), (iga2l.MIXED_FP32, 8, 132, "persistent"),
             (iga2l.MIXED_FP32, 6, 50, "lattice"), (iga2l.MIXED_FP32, 7, 40, "lattice"),
             (iga2l.MIXED_FP32, 8, 44, "lattice"),
             (iga2l.MIXED_FP32_ALL, 2, 50, "tile"), (iga2l.MIXED_FP32_ALL, 5, 70, "lattice_pc"),
             (iga2l.MIXED_FP32_ALL, 7, 40, "lattice"),
             (iga2l.MIXED_TF32, 2, 50, "lattice"), (iga2l.MIXED_TF32, 3, 64, "lattice"),
             (iga2l.MIXED_TF32, 4, 66, "lattice"), (iga2l.MIXED_TF32, 5, 70, "lattice"),
             (iga2l.MIXED_FP32, 2, 4, "lattice_pc"), (iga2l.MIXED_FP32, 5, 6, "tile"),
             (iga2l.MIXED_FP32, 6, 8, "work_list"), (iga2l.MIXED_FP32, 8, 10, "lattice"),
             (iga2l.MIXED_FP32_ALL, 4, 6, "tile")]


@pytest.mark.parametrize("precision,p,m,sched", MIXED_2D)
def test_mixed_2d_stays_inside_its_buffers(precision, p, m, sched):
    _run(lambda gd: _solver(p, m, gd, precision=precision, **_sched_kw(sched)), 600 + p)


@pytest.mark.parametrize("p,m,precision,sched", [
    (2, 12, iga2l.FP64, "lattice"), (3, 16, iga2l.FP64, "lattice"), (4, 20, iga2l.FP64, "lattice"),
    (2, 12, iga2l.FP64, "tile"), (3, 16, iga2l.FP64, "tile"), (4, 20, iga2l.FP64, "tile"),
    (3, 64, iga2l.MIXED_FP32, "lattice"), (3, 32, iga2l.MIXED_FP32, "tile"), (3, 32, iga2l.MIXED_FP32_ALL, "tile")])
def test_3d_stays_inside_its_buffers(p, m, precision, sched):
    kw = {"dim": 3, "precision": precision,
          "schedule": iga2l.SCHED_TILE if sched == "tile" else iga2l.SCHED_LATTICE}
    if p > 2:
        kw["period"], kw["stride"] = 7, 2
    _run(lambda gd: _solver(p, m, gd, **kw), 700 + p)


def _exercise_batch(S, mk, seed):
    N, nb = S.N, S.nbatch
    f = mk(np.concatenate([synth.coefficients(N, seed + k) for k in range(nb)]))
    f[N:2 * N] = 0.0   # one problem done before its first cycle
    u0 = np.concatenate([synth.initial_guess(N, seed + 50 + k) for k in range(nb)])
    out = {}
    b = mk(np.zeros(nb * N))
    S.rhs_from_coeffs(f, b)
    out["b"] = b
    d = mk(np.zeros(nb * N))
    S.residual(mk(u0), b, d)
    out["d"] = d
    u = mk(u0)
    S.schwarz_sweep(u, b)
    out["sweep"] = u
    u = mk(u0)
    S.cycle(u, b)
    out["cycle"] = u
    u = mk(u0)
    c, rel, _ = S.solve_batch(f, u, tol=1e-8, max_cycles=40)
    out["solve"], out["cycles"], out["rel"] = u, torch.tensor(c), torch.tensor(rel)
    return out


@pytest.mark.parametrize("p,m", [(3, 64), (2, 6)])
@pytest.mark.parametrize("precision,sched", [(iga2l.FP64, "lattice"), (iga2l.FP64, "tile"),
                                             (iga2l.MIXED_FP32, "tile"), (iga2l.MIXED_FP32, "work_list")])
def test_batch_stays_inside_its_buffers(p, m, precision, sched):
    _run(lambda gd: _solver(p, m, gd, nbatch=4, precision=precision, **_sched_kw(sched)), 800,
         exercise=_exercise_batch)


def test_guard_check_needs_the_flag():
    S = _solver(2, 24, False)
    with pytest.raises(iga2l.IgaError):
        S.guard_check()
