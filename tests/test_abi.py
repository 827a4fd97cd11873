"""CPU checks of the C ABI library: it loads, exports every symbol declared in
include/iga2l.h, and its host-side setup tables agree with the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2009_01499_gb300 import iga2l

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "iga2l.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(iga2l_[A-Za-z0-9_]+)\s*\(", hdr)))


def test_library_loads_and_exports_every_declared_symbol():
    lib = iga2l.load()
    declared = _declared_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(iga2l.EXPORTS) == declared


def test_error_strings_and_options():
    lib = iga2l.load()
    assert lib.iga2l_strerror(0) == b"ok"
    assert b"invalid" in lib.iga2l_strerror(-1)
    o = iga2l.default_options()
    assert o.precision == iga2l.FP64 and o.schedule == iga2l.SCHED_LATTICE
    assert o.coarse == iga2l.COARSE_VCYCLE and o.max_cycles == 100


def test_options_struct_layout_matches_the_header(tmp_path):
    """The binding's ctypes Options has the size and field offsets of iga2l_options."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in iga2l.Options._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "iga2l.h"\nint main(void){\n'
                   '  printf("%zu\\n", sizeof(iga2l_options));\n'
                   + "".join(f'  printf("%zu\\n", offsetof(iga2l_options, {f}));\n' for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(iga2l.Options)
    assert out[1:] == [getattr(iga2l.Options, f).offset for f in fields]
    o = iga2l.default_options()
    assert o.rhs == iga2l.RHS_COEFFS and o.test_flags == 0 and o.wait_budget_cycles == 0


def test_assemble_rejects_bad_arguments_before_touching_the_gpu():
    lib = iga2l.load()
    h = ctypes.c_void_p()
    # m odd, m < 4, m < p + 1 (2D); m < 4p + 4 in 3D
    for p, m, dim in [(1, 32, 2), (9, 64, 2), (2, 31, 2), (2, 2, 2), (8, 8, 2), (2, 32, 4), (3, 14, 3)]:
        rc = lib.iga2l_assemble(p, m, dim, None, ctypes.byref(h))
        assert rc in (iga2l.ERR_INVALID_ARG, iga2l.ERR_UNSUPPORTED)
        assert not h.value
    bad = iga2l.default_options(period=4)   # q < s + p
    assert lib.iga2l_assemble(2, 32, 2, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_INVALID_ARG
    bad = iga2l.default_options(period=6, stride=2)   # gcd(g, q) != 1
    assert lib.iga2l_assemble(2, 32, 2, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_INVALID_ARG
    for kw in ({"rhs": 2}, {"test_flags": 8}, {"wait_budget_cycles": -5}, {"sweep": 4}):
        bad = iga2l.default_options(**kw)
        assert lib.iga2l_assemble(2, 32, 2, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_INVALID_ARG, kw
        assert not h.value
    # the work-list sweep runs the 2D TILE schedule only
    bad = iga2l.default_options(sweep=iga2l.SWEEP_WORK_LIST)
    assert lib.iga2l_assemble(2, 32, 2, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_UNSUPPORTED
    bad = iga2l.default_options(sweep=iga2l.SWEEP_WORK_LIST, schedule=iga2l.SCHED_TILE)
    assert lib.iga2l_assemble(2, 16, 3, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_UNSUPPORTED
    assert not h.value
    # grids without interior blocks: no tensor-core form and no persistent sweep
    for kw in ({"precision": iga2l.MIXED_TF32}, {"precision": iga2l.MIXED_FP32, "sweep": iga2l.SWEEP_PERSISTENT}):
        bad = iga2l.default_options(**kw)
        assert lib.iga2l_assemble(3, 14, 2, ctypes.byref(bad), ctypes.byref(h)) == iga2l.ERR_UNSUPPORTED, kw
        assert not h.value


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("m", [12, 33])
def test_library_bands_match_oracle(oracle_mod, p, m):
    K, M = oracle_mod.assemble_1d(p, m)
    Kb, Mb = iga2l.host_bands(p, m)
    n = m + p - 2
    for i in range(n):
        for a in range(2 * p + 1):
            j = i + a - p
            ref_k = K[i, j] if 0 <= j < n else 0.0
            ref_m = M[i, j] if 0 <= j < n else 0.0
            # independent assemblies: rounding-level agreement (1e-13 relative to the row scale)
            assert abs(Kb[i, a] - ref_k) <= 1e-13 * m
            assert abs(Mb[i, a] - ref_m) <= 1e-13 / m


@pytest.mark.parametrize("p,m", [(p, m) for p in (2, 3, 4, 5) for m in (24, 40)] +
                         # the smallest grids of each degree (every block a boundary block)
                         [(2, 4), (3, 4), (4, 6), (5, 6), (6, 8), (7, 8), (8, 10), (8, 16)])
def test_library_restriction_matches_oracle(oracle_mod, p, m):
    R = oracle_mod.restriction_1d(p, m, aggressive=True)
    Rl = iga2l.host_restriction(p, m)
    assert np.array_equal(Rl == 0, R == 0)              # same band
    assert np.allclose(Rl, R, atol=1e-14, rtol=0)        # rounding-level agreement


def test_host_tables_refuse_grids_below_the_class_minimum():
    """n = m + p - 2 must be at least 2p - 1 (every boundary row class a row of the grid)."""
    lib = iga2l.load()
    R = np.zeros(64 * 64)
    for p, m in [(8, 8), (6, 6), (4, 4)]:
        assert m + p - 2 < 2 * p - 1
        rc = lib.iga2l_host_restriction(p, m, R.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        assert rc == iga2l.ERR_INVALID_ARG, (p, m)
