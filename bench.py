#!/usr/bin/env python
"""Benchmark of the multi-rhs HISQ CG hot path on one GB300 (or N, weak scaling).

Workload (the multi-rhs FP32 configuration): 32^3 x 8 lattice, synthetic
Haar-random fat links (0.9 x SU(3), r18) and Naik links (-1/24 x U(3), r14)
with staggered phases and an antiperiodic t boundary folded in, a bundle of
n = 8 complex Z2 sources, m = 0.01, mu = 0, even-odd system
(4m^2 - D_eo D_oe) x_e = b_e solved to a true relative residual of 1e-10
with FP32 inner iterations and FP64 reliable updates every 50 iterations.

One step = one complete hisq_cg_solve of the bundle with the gauge field
loaded and the sources resident in HBM. value = seconds per right-hand side
(whole job: wall time of the slowest rank / rhs solved by all ranks).

Also reported on the same JSON line:
  roofline      the multi-rhs Dslash (the dominant kernel): algorithmic bytes
                per launch / CUDA-event launch time vs the measured HBM peak
  dslash        the same Dslash as GB/s, GFlop/s (1146 flop/site/rhs) and
                fraction of 8 TB/s, plus an n sweep
  fp64          the plain FP64 single-rhs GPU CG on the same system, s/rhs
  e2e           the same solve through the C ABI with pinned host buffers
  cpu_baseline  the FP64 numpy oracle on the host cores (bounded sample)

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
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

METRIC = "multi-RHS Dslash HBM GB/s (frac of 8 TB/s); CG s/rhs to 1e-10, mixed vs FP64"
UNIT = "s/rhs"
L = (32, 32, 32, 8)
NRHS = 8
MASS = 0.01
TOL = 1e-10
RELIABLE_EVERY = 50
LINK_SEED = 1
SOURCE_SEED = 2
DSLASH_FLOPS_PER_SITE_RHS = 1146
L2_BYTES = 129 * 1024 * 1024
NOMINAL_HBM_GBS = 8000.0
# FP64 textbook CG iterations of this system (rhs 0) to 1e-10; written by
# oracle/cg_iterations.py, which runs the oracle only.
ITER_FILE = os.path.join(ROOT, "oracle", "cg_iterations_32x32x32x8_m0.01.json")


def workload_config(n_gpus: int) -> dict:
    return {
        "workload": "HISQ even-odd CG, 32^3x8, n=8 Z2 rhs, m=0.01, FP32 inner (U r18, N r14), "
                    "FP64 reliable updates every 50, tol 1e-10",
        "lattice": list(L), "nrhs_per_gpu": NRHS, "global_rhs": NRHS * n_gpus, "mass": MASS,
        "tol": TOL, "inner_prec": "f32", "recon_U": 18, "recon_N": 14,
        "reliable_every": RELIABLE_EVERY, "parallelism": f"rhs-bundle replicas x{n_gpus}",
        "l2": "inputs larger than L2 (134 MB of packed links) and L2 flushed between steps",
    }


def dslash_bytes_per_site(n: int, f_u: int, f_n: int, link_bytes: int, spinor_bytes: int) -> int:
    """Algorithmic bytes per output site: each link once, each vector in and out once."""
    return 8 * (f_u + f_n) * link_bytes + 12 * n * spinor_bytes


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; rhs bundles are independent)
# ---------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def source_seed_for_rank(rank: int) -> int:
    """Each rank solves its own bundle of sources: no data-path collective."""
    return SOURCE_SEED + 1000 * rank


def reduce_max(value: float, world: int, device=None) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="hisq_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, f[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# CPU oracle baseline (only this function and run_reference touch oracle/)
# ---------------------------------------------------------------------------

def fp64_iterations(default: int | None) -> tuple[int | None, str]:
    if os.path.exists(ITER_FILE):
        with open(ITER_FILE) as fh:
            return int(json.load(fh)["iterations"]), "oracle CG iteration count (oracle/cg_iterations.py)"
    return default, "iteration count of the FP64 GPU solve of the same system"


def oracle_sample(U, N, b1, iters: int) -> float:
    """Seconds per oracle CG iteration for one rhs on the full lattice."""
    from oracle import hisq_oracle as O
    t0 = time.perf_counter()
    O.cg(lambda q: O.apply_Ae(U, N, q, L, MASS), b1, tol=1e-300, maxiter=iters)
    return (time.perf_counter() - t0) / iters


def cpu_baseline(U, N, b, fp64_iters_gpu: int | None) -> dict:
    iters_total, how = fp64_iterations(fp64_iters_gpu)
    sample_iters = 3
    t_it = oracle_sample(U, N, b[:1], sample_iters)
    value = t_it * iters_total if iters_total else None
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": f"{sample_iters} iterations of the numpy FP64 oracle CG, 1 rhs on 32^3x8 "
                      f"({t_it:.3f} s/iteration), scaled by {iters_total} iterations ({how})"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    H.hisq.library()   # fails loudly if the CUDA library is missing

    U, N = gen.hisq_links(L, seed=LINK_SEED)
    b = gen.z2_source(L, NRHS, seed=source_seed_for_rank(rank))
    dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
    stream = torch.cuda.current_stream(dev)

    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g = H.hisq_gauge_load(L, dU, dN, prec=H.HISQ_F32, recon_U=18, recon_N=14)
    pack_s = time.perf_counter() - t0
    bt = [torch.from_numpy(b[k]).to(dev) for k in range(NRHS)]
    xt = [torch.zeros_like(t) for t in bt]
    params = H.cg_params(inner_prec=H.HISQ_F32, reliable_every=RELIABLE_EVERY)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        return H.hisq_cg_solve(g, MASS, 0.0, bt, xt, TOL, params, stream=stream)

    for _ in range(args.warmup):
        step()
    launches = 0
    durs = []
    stats_last = None
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        durs.append(e0.elapsed_time(e1) / 1e3)
        launches += 4 * st.total_iters + 4 * st.reliable_updates + 3
        stats_last = st
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    barrier(world)
    clocks = sampler.stop()
    t_step = sum(durs) / len(durs)
    t_step_max = reduce_max(t_step, world, dev)
    s_per_rhs = t_step_max / (NRHS * world)
    res = [stats_last.true_rel_res[k] for k in range(NRHS)]

    # ---- the dominant kernel alone: multi-rhs Dslash, FP32, U r18 / N r14 ----
    vh = int(np.prod(L)) // 2
    peaks = measured_peaks()

    def time_dslash(n, reps=40):
        vs = [torch.randn(vh, 3, dtype=torch.complex64, device=dev) for _ in range(n)]
        ws = [torch.empty_like(v) for v in vs]
        for _ in range(3):
            H.hisq_dslash(g, vs, ws, 0, H.HISQ_F32, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            H.hisq_dslash(g, vs, ws, 0, H.HISQ_F32, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        nbytes = dslash_bytes_per_site(n, 18, 14, 4, 4) * vh
        flops = DSLASH_FLOPS_PER_SITE_RHS * n * vh
        return t, nbytes, flops

    t_d, bytes_d, flops_d = time_dslash(NRHS)
    gbs = bytes_d / t_d / 1e9
    sweep = {}
    for n in (1, 2, 4, 16):
        tn, bn, fn = time_dslash(n, reps=20)
        sweep[str(n)] = {"us": round(tn * 1e6, 2), "gbs": round(bn / tn / 1e9, 1),
                         "gflops": round(fn / tn / 1e9, 1)}
    sweep[str(NRHS)] = {"us": round(t_d * 1e6, 2), "gbs": round(gbs, 1),
                        "gflops": round(flops_d / t_d / 1e9, 1)}

    # ---- end to end through the C ABI with pinned host buffers ----
    hb = [torch.from_numpy(b[k]).pin_memory() for k in range(NRHS)]
    hx = [torch.zeros_like(t).pin_memory() for t in hb]
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        H.hisq_cg_solve(g, MASS, 0.0, hb, hx, TOL, params, stream=stream)
    e2e_t = (time.perf_counter() - t0) / e2e_steps
    e2e_t = reduce_max(e2e_t, world, dev)
    bytes_in = sum(t.numel() * t.element_size() for t in hb)
    bytes_out = sum(t.numel() * t.element_size() for t in hx)

    # ---- plain FP64 single-rhs GPU CG on the same system (rank 0) ----
    fp64 = None
    fp64_iters = None
    if rank == 0:
        g64 = H.hisq_gauge_load(L, dU, dN, prec=H.HISQ_F64)
        x64 = [torch.zeros_like(bt[0])]
        p64 = H.cg_params(inner_prec=H.HISQ_F64)
        H.hisq_cg_solve(g64, MASS, 0.0, bt[:1], x64, TOL, p64, stream=stream)   # warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s64 = H.hisq_cg_solve(g64, MASS, 0.0, bt[:1], x64, TOL, p64, stream=stream)
        e1.record(stream)
        e1.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        fp64_iters = s64.total_iters
        diff = float(torch.linalg.vector_norm(x64[0] - xt[0]) / torch.linalg.vector_norm(x64[0]))
        fp64 = {"s_per_rhs": t64, "iterations": s64.total_iters,
                "true_rel_res": s64.true_rel_res[0],
                "mixed_over_fp64_time": s_per_rhs / t64,
                "mixed_vs_fp64_solution_rel_diff": diff}
        H.hisq_gauge_free(g64)

    out = {
        "metric": METRIC, "value": s_per_rhs, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step_max * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (Haar-random links, Z2 sources; seeded)",
        "config": workload_config(world),
        "cg": {"iterations": stats_last.total_iters, "reliable_updates": stats_last.reliable_updates,
               "max_true_rel_res": max(res), "wall_s_per_step": wall / args.steps},
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(gbs / peaks["hbm_gbs"], 4),
                     "traffic": None,
                     "kernel": "dslash_kernel<float,float,18,14,rpt,EPI_NONE> n=8 on 32^3x8",
                     "peak_source": peaks["source"],
                     "bytes_per_launch": bytes_d},
        "dslash": {"gbs": round(gbs, 1), "frac_of_8tbs": round(gbs / NOMINAL_HBM_GBS, 4),
                   "gflops": round(flops_d / t_d / 1e9, 1), "us_per_launch": round(t_d * 1e6, 2),
                   "sweep_n": sweep},
        "link_pack_s": pack_s,
        "fp64": fp64,
        "e2e": {"value": e2e_t / (NRHS * world), "unit": UNIT,
                "h2d_bytes_per_step": bytes_in, "d2h_bytes_per_step": bytes_out},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if rank == 0:
        try:
            out["cpu_baseline"] = cpu_baseline(U, N, b, fp64_iters)
        except Exception as e:   # the baseline never blocks the GPU number
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"failed: {e}"}
        print(json.dumps(out), flush=True)
    H.hisq_gauge_free(g)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import hisq_inputs as gen
    U, N = gen.hisq_links(L, seed=LINK_SEED)
    b = gen.z2_source(L, NRHS, seed=SOURCE_SEED)
    iters_total, how = fp64_iterations(None)
    per_step_iters = 1
    for _ in range(args.warmup):
        oracle_sample(U, N, b[:1], per_step_iters)
    ts = [oracle_sample(U, N, b[:1], per_step_iters) for _ in range(args.steps)]
    t_it = sum(ts) / len(ts)
    value = t_it * iters_total if iters_total else None
    sample = (f"{per_step_iters} numpy FP64 oracle CG iteration per step, 1 rhs on 32^3x8 "
              f"({t_it:.3f} s/iteration), scaled by {iters_total} iterations ({how})")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * per_step_iters * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Haar-random links, Z2 sources; seeded)", "config": workload_config(world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
