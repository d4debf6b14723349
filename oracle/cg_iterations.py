"""Iteration count of the oracle's FP64 CG on the 32^3x8 benchmark system.

Runs the textbook CG of ``hisq_oracle`` (test infrastructure) on
(4m^2 - D_eo D_oe) x = b with m = 0.01, links seed 1, the first Z2 source of
seed 2, until the relative residual is 1e-10, and writes the count to
cg_iterations_32x32x32x8_m0.01.json beside this file. The CPU baseline of
bench.py multiplies a timed sample of oracle iterations by this count to
express the oracle in seconds per rhs. Takes about an hour on one core.

    python -m oracle.cg_iterations
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import hisq_inputs as gen  # noqa: E402
from oracle import hisq_oracle as O  # noqa: E402

L = (32, 32, 32, 8)
MASS = 0.01
TOL = 1e-10
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cg_iterations_32x32x32x8_m0.01.json")


def main():
    U, N = gen.hisq_links(L, seed=1)
    b = gen.z2_source(L, 8, seed=2)[:1]
    t0 = time.perf_counter()
    x, iters = O.cg(lambda q: O.apply_Ae(U, N, q, L, MASS), b, tol=TOL)
    dt = time.perf_counter() - t0
    res = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, MASS), x, b)
    rec = {"lattice": list(L), "mass": MASS, "tol": TOL, "link_seed": 1, "source_seed": 2,
           "rhs": 0, "iterations": int(iters[0]), "true_rel_res": float(res[0]),
           "seconds": dt, "seconds_per_iteration": dt / max(1, int(iters[0]))}
    with open(OUT, "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
