"""Writes oracle_cycles_m1024.json: the oracle's own cycle counts to a 1e-8 relative
residual on the benchmark workload (2D, p = 2..5, 1024x1024 elements, seeded
uniform[-1,1] coefficients of f, seeded uniform[-1,1] initial guess, LATTICE
colouring, aggressive 2h second level with one V(1,1) cycle).

Calls only oracle/ (and the seeded input generator).  The benchmark's reference
arm times single oracle cycles and scales them by these counts.
Run from the repository root: python tests/golden/make_oracle_cycles.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2009_01499_gb300 import synth  # noqa: E402

M = 1024
COLOURING = {2: (5, 2), 3: (7, 2), 4: (7, 2), 5: (10, 3)}


def main():
    out = {"_what": __doc__.strip().splitlines()[0], "m": M, "tol": 1e-8, "cycles": {}, "seeds": {}}
    for p in (2, 3, 4, 5):
        q, g = COLOURING[p]
        O = oracle.Problem(2, p, M, sched=oracle.LATTICE, coarse=oracle.VCYCLE, period=q, stride=g)
        seed = synth.BASE_SEED + 1
        f = synth.coefficients(O.N, seed + p)
        u0 = synth.initial_guess(O.N, seed + 10 + p)
        K, Mm = oracle.assemble_1d(p, M)
        b = (Mm @ f.reshape(O.n, O.n) @ Mm.T).ravel()
        t = time.time()
        _, cyc, rel, hist, ok = O.solve(b, u0, tol=1e-8, maxc=60)
        assert ok
        out["cycles"][str(p)] = cyc
        out["seeds"][str(p)] = {"f": seed + p, "u0": seed + 10 + p}
        print(f"p={p}: {cyc} cycles, rel {rel:.3e}, {time.time() - t:.1f}s", flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_cycles_m1024.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
