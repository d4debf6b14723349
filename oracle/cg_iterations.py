"""Iteration count of the oracle's FP64 CG on a benchmark system.

Runs the textbook CG of ``hisq_oracle`` (test infrastructure) on
(4m^2 - D_eo D_oe) x = b with links seed 1 and the first source of seed 2
until the relative residual is 1e-10, and writes the count to
cg_iterations_<lattice>_m<mass>.json beside this file. The CPU baseline of
bench.py multiplies a timed sample of oracle iterations by this count to
express the oracle in seconds per rhs. Two systems:

    python -m oracle.cg_iterations                  # 32^3x8, m = 0.01, Z2 source (about an hour)
    python -m oracle.cg_iterations --mixed          # 48^3x12, m = 0.0025, Gaussian source (many hours)
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import hisq_inputs as gen  # noqa: E402
from oracle import hisq_oracle as O  # noqa: E402

TOL = 1e-10
SYSTEMS = {
    "fp32": ((32, 32, 32, 8), 0.01, "z2"),
    "mixed": ((48, 48, 48, 12), 0.0025, "gaussian"),
}


def out_path(L, mass):
    lat = "x".join(str(a) for a in L)
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), f"cg_iterations_{lat}_m{mass}.json")


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--mixed", action="store_true", help="the 48^3x12 light-mass system")
    a = ap.parse_args(argv)
    L, mass, kind = SYSTEMS["mixed" if a.mixed else "fp32"]
    U, N = gen.hisq_links(L, seed=1)
    src = gen.gaussian_source if kind == "gaussian" else gen.z2_source
    b = src(L, 8, seed=2)[:1]
    t0 = time.perf_counter()
    x, iters = O.cg(lambda q: O.apply_Ae(U, N, q, L, mass), b, tol=TOL)
    dt = time.perf_counter() - t0
    res = O.true_relative_residual(lambda q: O.apply_Ae(U, N, q, L, mass), x, b)
    rec = {"lattice": list(L), "mass": mass, "tol": TOL, "link_seed": 1, "source_seed": 2,
           "source": kind, "rhs": 0, "iterations": int(iters[0]), "true_rel_res": float(res[0]),
           "seconds": dt, "seconds_per_iteration": dt / max(1, int(iters[0]))}
    with open(out_path(L, mass), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
