"""GPU test of iga2l_residual_norm2_noalloc, the entry point for callers that
cannot allocate device memory (they cannot create a solver handle, because
iga2l_assemble allocates).  It is checked through the C ABI against the
handle-based iga2l_residual on two calls in a row, with different inputs, so
that anything left over in the shared fixed scratch from the first call would
show up in the second.  Kept in its own file, collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2009_01499_gb300 import iga2l, synth  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def test_noalloc_residual_matches_handle_entry_point_twice():
    for p, m, seed in [(3, 100, 11), (5, 70, 12)]:
        S = iga2l.Solver(p, m)
        K, M = iga2l.host_bands(p, m)
        Kd, Md = _dev(K.ravel()), _dev(M.ravel())
        for call, s in enumerate((seed, seed + 100)):
            u = _dev(synth.initial_guess(S.N, s))
            b = _dev(synth.coefficients(S.N, s + 1))
            d_ref = torch.empty_like(u)
            nrm_ref = S.residual(u, b, d_ref, want_norm=True)
            d = torch.full_like(u, float("nan"))
            norm2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            iga2l.residual_norm2_noalloc(p, S.n, Kd, Md, u, b, d, norm2)
            torch.cuda.synchronize()
            got = float(norm2.item()) ** 0.5
            assert abs(got - nrm_ref) <= TOL * nrm_ref, (p, call, got, nrm_ref)
            dr = d_ref.cpu().numpy()
            assert np.abs(d.cpu().numpy() - dr).max() <= TOL * np.abs(dr).max(), (p, call)
        S.close()


def test_noalloc_norm_only_and_largest_grid():
    """d = NULL (norm only) against the handle's norm, and n = 4096 (the largest grid the
    fixed scratch takes: exactly 65536 partial sums) against iga2l_residual."""
    for p, m, want_d in [(4, 90, False), (2, 4096, True)]:
        S = iga2l.Solver(p, m)
        assert S.n <= 4096
        K, M = iga2l.host_bands(p, m)
        Kd, Md = _dev(K.ravel()), _dev(M.ravel())
        u = _dev(synth.initial_guess(S.N, 31))
        b = _dev(synth.coefficients(S.N, 32))
        d_ref = torch.empty_like(u) if want_d else None
        nrm_ref = S.residual(u, b, d_ref, want_norm=True)
        d = torch.full_like(u, float("nan")) if want_d else None
        norm2 = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        iga2l.residual_norm2_noalloc(p, S.n, Kd, Md, u, b, d, norm2)
        torch.cuda.synchronize()
        got = float(norm2.item()) ** 0.5
        assert abs(got - nrm_ref) <= TOL * nrm_ref, (p, m, got, nrm_ref)
        if want_d:
            dr = d_ref.cpu().numpy()
            assert np.abs(d.cpu().numpy() - dr).max() <= TOL * np.abs(dr).max(), (p, m)
        S.close()
        del u, b, d, d_ref
        torch.cuda.empty_cache()


def test_noalloc_rejects_oversized_grid_with_clear_error():
    lib = iga2l.load()
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = lib.iga2l_residual_norm2_noalloc(2, 5000, one.data_ptr(), one.data_ptr(), one.data_ptr(),
                                          one.data_ptr(), None, one.data_ptr(), None)
    assert rc == iga2l.ERR_INVALID_ARG
    assert b"4096" in lib.iga2l_last_error()
    for n in (4097, 2 ** 31 - 1):   # one past the limit; and near INT_MAX (no wrap-around)
        rc = lib.iga2l_residual_norm2_noalloc(2, n, one.data_ptr(), one.data_ptr(), one.data_ptr(),
                                              one.data_ptr(), None, one.data_ptr(), None)
        assert rc == iga2l.ERR_INVALID_ARG, n
        assert b"4096" in lib.iga2l_last_error()
