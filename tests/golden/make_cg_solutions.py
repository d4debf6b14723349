"""Oracle CG solutions of the configurations' systems, sampled, for the GPU parity tests.

Runs the FP64 textbook CG of ``oracle.hisq_oracle`` (nothing else computes
here) on the even-odd system (4m^2 - D_eo D_oe) x = b of each case below to
an iterated relative residual of 1e-13, and stores, per rhs, the full
solution norm, the oracle's true relative residual and a seeded sample of
solution components (site, colour) in ``cg_solution_<case>.npz`` beside this
file. The GPU tests solve the same systems and compare the sampled components
element by element (solution relative error <= 1e-8 at true residual <= 1e-10).

Cases (links seed 1 of hisq_inputs; sources seed 2):
  light16    16^4, m = 0.0025, 4 Gaussian sources (the mixed-precision
             configuration's mass; about 14600 iterations, 4.6 hours on one
             core)
  light8     8^4, m = 0.0025, 4 Gaussian sources
  fp32cfg    16^3x8, m = 0.01, 8 complex Z2 sources (the multi-rhs FP32
             configuration's mass and bundle)

    python tests/golden/make_cg_solutions.py [case ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import hisq_inputs as gen  # noqa: E402
from oracle import hisq_oracle as O  # noqa: E402

CASES = {
    "light16": ((16, 16, 16, 16), 0.0025, "gaussian", 4),
    "light8": ((8, 8, 8, 8), 0.0025, "gaussian", 4),
    "fp32cfg": ((16, 16, 16, 8), 0.01, "z2", 8),
}
SAMPLES = 2048          # sampled components per rhs
ORACLE_TOL = 1e-13


def path(case):
    return os.path.join(HERE, f"cg_solution_{case}.npz")


def sources(L, kind, n):
    src = gen.gaussian_source if kind == "gaussian" else gen.z2_source
    return src(L, n, seed=2)


def sample_index(L, n):
    """Seeded (rhs, site, colour) sample: the same for the writer and the tests."""
    vh = int(np.prod(L)) // 2
    rng = np.random.default_rng(12345)
    return rng.integers(0, vh, size=(n, SAMPLES)), rng.integers(0, 3, size=(n, SAMPLES))


def make(case):
    L, mass, kind, n = CASES[case]
    U, N = gen.hisq_links(L, seed=1)
    b = sources(L, kind, n)

    def A(q):
        return O.apply_Ae(U, N, q, L, mass)

    t0 = time.perf_counter()
    x, iters = O.cg(A, b, tol=ORACLE_TOL)
    dt = time.perf_counter() - t0
    res = O.true_relative_residual(A, x, b)
    site, colour = sample_index(L, n)
    vals = np.stack([x[k, site[k], colour[k]] for k in range(n)])
    np.savez(path(case), values=vals, site=site, colour=colour,
             norm=np.linalg.norm(x.reshape(n, -1), axis=1), true_rel_res=res,
             iterations=np.asarray(iters), lattice=np.asarray(L), mass=mass)
    print(json.dumps({"case": case, "lattice": list(L), "mass": mass, "n": n,
                      "iterations": [int(i) for i in iters], "true_rel_res": [float(r) for r in res],
                      "seconds": dt}), flush=True)


if __name__ == "__main__":
    for c in (sys.argv[1:] or list(CASES)):
        make(c)
