"""Run a fixed number of multi-rhs Dslash (or CG) launches for profiling.

A small, self-contained driver for `ncu` captures and event timing of one
kernel configuration, outside the benchmark:

    python -m paper_1411_4439_gb300.dslash_probe --lattice 48 48 48 12 --n 8 \\
        --prec f32 --recon 18 14 --reps 3

Prints one JSON line with the CUDA-event time per launch and the
algorithmic GB/s (8 (f_U + f_N) s_l + 12 n s_s bytes per output site).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PREC = {"f64": 0, "f32": 1, "f16": 2}
BYTES = {"f64": 8, "f32": 4, "f16": 2}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--lattice", type=int, nargs=4, default=[48, 48, 48, 12])
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--prec", choices=sorted(PREC), default="f32")
    ap.add_argument("--recon", type=int, nargs=2, default=[18, 14])
    ap.add_argument("--rpt", type=int, default=0)
    ap.add_argument("--minb", type=int, default=0)
    ap.add_argument("--pack", type=int, default=0)
    ap.add_argument("--prefetch", type=int, default=0)
    ap.add_argument("--staged", type=int, default=0, help="4 = links staged in shared memory")
    ap.add_argument("--pipe", type=int, default=0, help="1 or 2: loads of the next 1 or 2 hops in flight")
    ap.add_argument("--layout", choices=["aos", "soa"], default="soa")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--op", choices=["dslash", "mdagm"], default="dslash")
    a = ap.parse_args(argv)

    import numpy as np
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H

    L = tuple(a.lattice)
    prec = PREC[a.prec]
    U, N = gen.hisq_links(L, seed=1)
    dev = torch.device("cuda", 0)
    g = H.hisq_gauge_load(L, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev), prec=prec,
                          recon_U=a.recon[0] if prec else 18, recon_N=a.recon[1] if prec else 18)
    del U, N
    if a.rpt or a.pack or a.prefetch or a.staged or a.pipe:
        pipe = {0: 0, 1: H.hisq.HISQ_MAP_PIPELINED, 2: H.hisq.HISQ_MAP_PIPELINED2}[a.pipe]
        H.hisq_set_dslash_mapping(g, a.rpt, a.minb, a.pack * H.hisq.HISQ_MAP_PACKED
                                  + a.prefetch * H.hisq.HISQ_MAP_L2_PREFETCH
                                  + (H.hisq.HISQ_MAP_STAGED if a.staged else 0) + pipe)
    mapping = H.hisq_get_dslash_mapping(g, a.n, prec)
    vh = int(np.prod(L)) // 2
    if a.prec == "f64":
        vs = [torch.randn(vh, 3, dtype=torch.complex128, device=dev) for _ in range(a.n)]
    elif a.prec == "f32":
        vs = [torch.randn(vh, 3, dtype=torch.complex64, device=dev) for _ in range(a.n)]
    else:
        vs = [torch.randn(vh, 3, 2, device=dev).half() for _ in range(a.n)]
    ws = [torch.empty_like(v) for v in vs]
    layout = H.HISQ_SOA if a.layout == "soa" else H.HISQ_AOS
    stream = torch.cuda.current_stream(dev)

    def launch():
        if a.op == "dslash":
            H.hisq_dslash_ex(g, 0.0, vs, ws, 0, prec, layout, stream=stream)
        else:
            H.hisq_mdagm(g, 0.01, vs, ws, prec, stream=stream)

    for _ in range(a.warmup):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.reps):
        launch()
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / a.reps
    fu = 18 if prec == 0 else a.recon[0]
    fn = 18 if prec == 0 else a.recon[1]
    nb = (8 * (fu + fn) * BYTES[a.prec] + 12 * a.n * BYTES[a.prec]) * vh
    ops = 2 if a.op == "mdagm" else 1
    print(json.dumps({"lattice": L, "n": a.n, "prec": a.prec, "recon": [fu, fn], "op": a.op,
                      "rpt": mapping[0], "minb": mapping[1], "flags": mapping[2],
                      "staged": bool(mapping[2] & H.hisq.HISQ_MAP_STAGED),
                      "pack": a.pack, "prefetch": a.prefetch, "pipe": a.pipe,
                      "layout": a.layout,
                      "us_per_launch": t * 1e6 / ops, "alg_bytes_per_dslash": nb,
                      "alg_gbs": nb * ops / t / 1e9, "gflops": 1146 * a.n * vh * ops / t / 1e9}))
    H.hisq_gauge_free(g)


if __name__ == "__main__":
    main()
