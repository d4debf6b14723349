#!/usr/bin/env python
"""Benchmark of the multi-rhs HISQ CG hot path on one GB300 (or N, weak scaling).

Workload (the mixed-precision multi-rhs configuration): 48^3 x 12 lattice,
synthetic Haar-random fat links (0.9 x SU(3), stored in 18 reals) and Naik
links (-1/24 x U(3), 14 reals) with staggered phases and an antiperiodic t
boundary folded in, all link reals stored as 16-bit fixed point, a bundle of
n = 8 Gaussian complex sources, m = 0.0025, mu = 0, even-odd system
(4m^2 - D_eo D_oe) x_e = b_e solved to a true relative residual of 1e-10 with
FP16 spinor storage and FP32 arithmetic in the inner iteration, FP64
reliable updates every 150 iterations (true residual with FP64 links) and an
FP64 solution.

One step = one complete hisq_cg_solve of the bundle with the gauge field
loaded and the sources resident in HBM. value = seconds per right-hand side
(whole job: wall time of the slowest rank / rhs solved by all ranks).

Also reported on the same JSON line:
  roofline      the FP16 multi-rhs Dslash of the solve (the dominant kernel):
                algorithmic flops (bytes) per launch / CUDA-event launch time
                against the FP32 ALU peak (the measured HBM peak), L2 flushed
                between launches
  dslash        the same Dslash, and the FP32-storage one, as GB/s, GFlop/s
                (1146 flop/site/rhs) and fractions of both peaks
  fp64          the plain FP64 single-rhs GPU CG on the same system and
                source 0 (the comparison of "mixed vs FP64"), s/rhs
  cg_kernels    the four launches of an iteration of the same solve timed hot
                (CUDA events around each launch, hisq_cg_params.profile_kernels)
                against their byte minima
  configs1      the multi-rhs FP32 configuration (32^3x8, n = 8, m = 0.01)
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
# the headline workload: mixed precision, 48^3x12
L = (48, 48, 48, 12)
NRHS = 8
MASS = 0.0025
TOL = 1e-10
# FP64 reliable update every 150 iterations: at 48^3x12, m = 0.0025 a solve of
# 8 rhs took 7.76 / 7.59 / 7.50 / 7.57 / 8.61 s at 100 / 125 / 150 / 200 / 300
# (fewer iterations against more FP64 updates); at 400 it did not converge
RELIABLE_EVERY = 150
# the multi-rhs FP32 configuration (reported beside the headline)
L1 = (32, 32, 32, 8)
MASS1 = 0.01
RELIABLE_EVERY1 = 50
LINK_SEED = 1
SOURCE_SEED = 2
DSLASH_FLOPS_PER_SITE_RHS = 1146
L2_BYTES = 129 * 1024 * 1024
NOMINAL_HBM_GBS = 8000.0
# FP32 lanes of one SM and its clock: the FP32 ALU peak is SMs x 128 x 2 flop x clock
FP32_LANES_PER_SM = 128
# FP64 textbook CG iterations of the 32^3x8 system (rhs 0) to 1e-10; written
# by oracle/cg_iterations.py, which runs the oracle only.
ITER_FILE = os.path.join(ROOT, "oracle", "cg_iterations_32x32x32x8_m0.01.json")


def workload_config(n_gpus: int) -> dict:
    return {
        "workload": "HISQ even-odd CG, 48^3x12, n=8 Gaussian rhs, m=0.0025, FP16 storage (16-bit "
                    "fixed-point links U r18 / N r14, half spinors) with FP32 arithmetic, FP64 reliable "
                    f"updates every {RELIABLE_EVERY} and FP64 solution, tol 1e-10",
        "lattice": list(L), "nrhs_per_gpu": NRHS, "global_rhs": NRHS * n_gpus, "mass": MASS,
        "tol": TOL, "inner_prec": "f16 storage, f32 arithmetic", "storage_dtype": "f16",
        "recon_U": 18, "recon_N": 14, "reliable_every": RELIABLE_EVERY,
        "spinor_layout": "bundle", "parallelism": f"rhs-bundle replicas x{n_gpus}",
        "l2": "inputs larger than L2 (340 MB of packed links, 1.5 GB FP64 links) and L2 flushed between steps",
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


# DRAM bytes (read + write) of one launch of a roofline Dslash, from one ncu
# capture of that kernel (profiles/), keyed by (precision, lattice, n, rhs per
# thread, min blocks, mapping flags). A mapping without a capture reports null.
DSLASH_TRAFFIC = {
    # profiles/dslash_bundle_f16_r18_r14_n8_48x48x48x12.md: 418.9 MB read + 37.1 MB written
    ("f16", (48, 48, 48, 12), 8, 8, 4, 132): 455975424,
    # profiles/dslash_bundle_f32_r18_r14_n8_48x48x48x12.md: 831.5 MB read + 100.1 MB written
    ("f32", (48, 48, 48, 12), 8, 8, 3, 0): 931567104,
}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


def fp32_peak_tflops(sm_count: int, mhz: float) -> float:
    """FP32 ALU peak: every SM retires 128 fused multiply-adds (2 flop) per clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def roofline_bound(flops: float, nbytes: float, alu_tflops: float, hbm_gbs: float) -> str:
    """The roofline that binds a kernel: "alu" when its arithmetic intensity
    lies past the ridge (ALU peak / HBM peak), else "hbm"."""
    return "alu" if flops / nbytes > alu_tflops * 1e3 / hbm_gbs else "hbm"


def dslash_traffic(prec: str, lattice, n: int, mapping) -> int | None:
    """ncu DRAM bytes of one launch of a captured Dslash configuration, else None."""
    return DSLASH_TRAFFIC.get((prec, tuple(lattice), n) + tuple(mapping))


# ---------------------------------------------------------------------------
# CPU oracle baseline (only this function and run_reference touch oracle/)
# ---------------------------------------------------------------------------

def fp64_iterations(default: int | None, mixed: bool = False) -> tuple[int | None, str]:
    """The oracle's own FP64 CG iteration count of the system if it has been
    written (oracle/cg_iterations.py), else the given count."""
    name = "cg_iterations_48x48x48x12_m0.0025.json" if mixed else "cg_iterations_32x32x32x8_m0.01.json"
    path = os.path.join(ROOT, "oracle", name)
    if os.path.exists(path):
        with open(path) as fh:
            return int(json.load(fh)["iterations"]), "oracle CG iteration count (oracle/cg_iterations.py)"
    return default, "iteration count of the FP64 GPU solve of the same system"


def oracle_sample(U, N, b1, iters: int) -> float:
    """Seconds per oracle CG iteration for one rhs of the headline system."""
    from oracle import hisq_oracle as O
    t0 = time.perf_counter()
    O.cg(lambda q: O.apply_Ae(U, N, q, L, MASS), b1, tol=1e-300, maxiter=iters)
    return (time.perf_counter() - t0) / iters


def cpu_baseline(U, N, b, fp64_iters_gpu: int | None) -> dict:
    iters_total, how = fp64_iterations(fp64_iters_gpu, mixed=True)
    sample_iters = 3
    t_it = oracle_sample(U, N, b[:1], sample_iters)
    value = t_it * iters_total if iters_total else None
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "host_cpus": os.cpu_count(),
            "sample": f"{sample_iters} iterations of the numpy FP64 oracle CG, 1 rhs on 48^3x12 "
                      f"({t_it:.3f} s/iteration), scaled by {iters_total} iterations ({how})"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def time_bundle_dslash(H, torch, g, prec, n, stream, flush, reps=20):
    """Per-launch CUDA-event time (mean over reps) of the bundle Dslash the CG
    uses, with an L2 flush (a write larger than L2) before every launch."""
    vh = int(np.prod(g.L)) // 2
    dt = torch.float32 if prec == H.HISQ_F32 else torch.float16
    src = [torch.randn(vh, 3, dtype=torch.complex128, device=flush.device) for _ in range(n)]
    vb = torch.empty(H.hisq.bundle_bytes(g, n, prec) // (4 if prec == H.HISQ_F32 else 2), dtype=dt,
                     device=flush.device)
    H.hisq_bundle_pack(g, src, prec, vb, stream=stream)
    del src
    wb = torch.empty_like(vb)
    for _ in range(3):
        H.hisq_dslash_ex(g, 0.0, vb, wb, 0, prec, H.HISQ_BUNDLE, stream=stream, n=n)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        flush.fill_(1.0)
        e0.record(stream)
        H.hisq_dslash_ex(g, 0.0, vb, wb, 0, prec, H.HISQ_BUNDLE, stream=stream, n=n)
        e1.record(stream)
    torch.cuda.synchronize()
    t = sum(e0.elapsed_time(e1) for e0, e1 in ev) / 1e3 / reps
    sb = 4 if prec == H.HISQ_F32 else 2
    nbytes = dslash_bytes_per_site(n, g.recon_U, g.recon_N, sb, sb) * vh
    flops = DSLASH_FLOPS_PER_SITE_RHS * n * vh
    return t, nbytes, flops


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
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    peaks = measured_peaks()
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = fp32_peak_tflops(sm_count, peaks["sm_max_mhz"])

    U, N = gen.hisq_links(L, seed=LINK_SEED)
    b = gen.gaussian_source(L, NRHS, seed=source_seed_for_rank(rank))
    dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    g = H.hisq_gauge_load(L, dU, dN, prec=H.HISQ_F16, recon_U=18, recon_N=14)
    pack_s = time.perf_counter() - t0
    bt = [torch.from_numpy(b[k]).to(dev) for k in range(NRHS)]
    xt = [torch.zeros_like(t) for t in bt]
    params = H.cg_params(inner_prec=H.HISQ_F16, reliable_every=RELIABLE_EVERY,
                         spinor_layout=H.HISQ_BUNDLE)

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
        # per iteration: two Dslash, update_r, update_px; per reliable update:
        # accumulate, two FP64 Dslash, best-iterate copy, rescale; per solve:
        # norm |b|, copy the residual, best-iterate copy, rescale; per chunk
        # of check_every iterations of the device-driven loop: the decision
        # and booking kernels
        chunks = -(-st.total_iters // params.check_every)
        launches += 4 * st.total_iters + 5 * st.reliable_updates + 4 + 2 * chunks
        stats_last = st
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    barrier(world)
    clocks = sampler.stop()
    t_step = sum(durs) / len(durs)
    t_step_max = reduce_max(t_step, world, dev)
    s_per_rhs = t_step_max / (NRHS * world)
    res = [stats_last.true_rel_res[k] for k in range(NRHS)]

    # ---- the dominant kernel alone: FP16 bundle Dslash of the solve, and FP32 ----
    t_d, bytes_d, flops_d = time_bundle_dslash(H, torch, g, H.HISQ_F16, NRHS, stream, flush)
    mapping = H.hisq_get_dslash_mapping_ex(g, NRHS, H.HISQ_F16, H.HISQ_BUNDLE)
    gbs = bytes_d / t_d / 1e9
    tfl = flops_d / t_d / 1e12
    intensity = flops_d / bytes_d
    ridge = alu_peak * 1e3 / peaks["hbm_gbs"]
    kernel_d = (f"dslash_bundle_kernel<__half,Fx16,18,14,rpt={mapping[0]},minb={mapping[1]},"
                f"flags={mapping[2]}> n={NRHS} on 48x48x48x12")
    traffic_d = dslash_traffic("f16", L, NRHS, mapping)
    hbm = {"achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": round(gbs / peaks["hbm_gbs"], 4), "peak_source": peaks["source"]}
    alu = {"achieved": round(tfl, 2), "peak": round(alu_peak, 1), "unit": "TFLOP/s",
           "frac": round(tfl / alu_peak, 4),
           "peak_source": f"derived: {sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                          f"{peaks['sm_max_mhz']:.0f} MHz"}
    bound = roofline_bound(flops_d, bytes_d, alu_peak, peaks["hbm_gbs"])
    main = alu if bound == "alu" else hbm
    dslash_info = {"f16": {"us_per_launch": round(t_d * 1e6, 2), "gbs": round(gbs, 1),
                           "frac_of_8tbs": round(gbs / NOMINAL_HBM_GBS, 4), "hbm_frac": hbm["frac"],
                           "tflops": round(tfl, 2), "alu_frac": alu["frac"],
                           "flop_per_byte": round(intensity, 2), "mapping": list(mapping),
                           "traffic": traffic_d}}
    g32 = H.hisq_gauge_load(L, dU, dN, prec=H.HISQ_F32, recon_U=18, recon_N=14)
    t32, b32, f32 = time_bundle_dslash(H, torch, g32, H.HISQ_F32, NRHS, stream, flush)
    dslash_info["f32"] = {"us_per_launch": round(t32 * 1e6, 2), "gbs": round(b32 / t32 / 1e9, 1),
                          "hbm_frac": round(b32 / t32 / 1e9 / peaks["hbm_gbs"], 4),
                          "tflops": round(f32 / t32 / 1e12, 2),
                          "alu_frac": round(f32 / t32 / 1e12 / alu_peak, 4),
                          "flop_per_byte": round(f32 / b32, 2),
                          "mapping": list(H.hisq_get_dslash_mapping_ex(g32, NRHS, H.HISQ_F32,
                                                                                 H.HISQ_BUNDLE))}
    dslash_info["f32"]["traffic"] = dslash_traffic("f32", L, NRHS, dslash_info["f32"]["mapping"])
    H.hisq_gauge_free(g32)
    cg_kernels = time_cg_kernels(H, torch, g, bt, params, stream)

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

    # ---- plain FP64 single-rhs GPU CG on the same system and source 0 (rank 0) ----
    fp64 = None
    fp64_iters = None
    configs1 = None
    if rank == 0:
        g64 = H.hisq_gauge_load(L, dU, dN, prec=H.HISQ_F64)
        x64 = [torch.zeros_like(bt[0])]
        p64 = H.cg_params(inner_prec=H.HISQ_F64)
        try:   # warm-up: a few iterations (workspace, graphs)
            H.hisq_cg_solve(g64, MASS, 0.0, bt[:1], x64, TOL, H.cg_params(inner_prec=H.HISQ_F64, maxiter=20),
                            stream=stream)
        except H.HisqError:
            pass
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
        del x64
        configs1 = run_configs1(H, torch, gen, dev, stream)
    del dU, dN

    out = {
        "metric": METRIC, "value": s_per_rhs, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step_max * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (Haar-random links, Gaussian sources; seeded)",
        "config": workload_config(world),
        "cg": {"iterations": stats_last.total_iters, "reliable_updates": stats_last.reliable_updates,
               "max_true_rel_res": max(res), "wall_s_per_step": wall / args.steps},
        "roofline": dict(main, bound=bound, traffic=traffic_d, kernel=kernel_d,
                         bytes_per_launch=bytes_d, flops_per_launch=flops_d, hbm=hbm, alu=alu,
                         ridge_flop_per_byte=round(ridge, 2)),
        "dslash": dslash_info,
        "cg_kernels": cg_kernels,
        "link_pack_s": pack_s,
        "fp64": fp64,
        "configs1": configs1,
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


def cg_kernel_byte_minima(vh: int, n: int) -> dict:
    """Byte minima of the four launches of an FP16-storage CG iteration (U r18,
    N r14 16-bit links, half spinors, FP32 solution increment), V_h sites."""
    sp = 12 * n               # FP16 spinor bytes per site
    xl = 24 * n               # FP32 x_lo bytes per site
    links = 8 * (18 + 14) * 2
    return {"dslash_t": (links + 2 * sp) * vh,            # t = D_oe p
            "dslash_ap_alpha": (links + 3 * sp) * vh,     # Ap = 4m^2 p - D_eo t (reads p), Re<p, Ap>
            "update_r": 3 * sp * vh,                      # r, Ap in; r out
            "update_px": (3 * sp + 2 * xl) * vh}          # p, x_lo, r in; x_lo, p out


def time_cg_kernels(H, torch, g, bt, params, stream, iters: int = 400) -> dict:
    """The four launches of a CG iteration of the headline solve, timed hot
    with CUDA events on the solve's stream (hisq_cg_params.profile_kernels)
    over the first `iters` iterations, against their byte minima: per site,
    FP16 spinors of 8 rhs are 96 B and the FP32 solution increment 192 B."""
    minima = cg_kernel_byte_minima(int(np.prod(L)) // 2, NRHS)
    p = H.cg_params(inner_prec=params.inner_prec, reliable_every=params.reliable_every,
                    spinor_layout=params.spinor_layout, maxiter=iters, profile_kernels=1)
    x = [torch.zeros_like(t) for t in bt]
    try:
        st = H.hisq_cg_solve(g, MASS, 0.0, bt, x, TOL, p, stream=stream)
    except H.HisqError as e:     # HISQ_ENOCONV at the cap: the stats ride on the error
        st = e.stats
    peak = measured_peaks()["hbm_gbs"]
    out = {"iterations_timed": st.profiled_iters}
    for k, name in enumerate(minima):
        us = st.kernel_us[k]
        gbs = minima[name] / (us * 1e-6) / 1e9 if us > 0 else None
        out[name] = {"us": round(us, 2), "min_bytes": minima[name],
                     "gbs": None if gbs is None else round(gbs, 1),
                     "hbm_frac": None if gbs is None else round(gbs / peak, 4)}
    return out


def run_configs1(H, torch, gen, dev, stream) -> dict:
    """The multi-rhs FP32 configuration beside the headline: 32^3x8, n = 8 Z2
    sources, m = 0.01, FP32 storage (U r18 / N r14), FP64 reliable updates
    every 50; one timed solve after a warm-up, and the FP64 single-rhs solve."""
    U, N = gen.hisq_links(L1, seed=LINK_SEED)
    dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
    b = gen.z2_source(L1, NRHS, seed=SOURCE_SEED)
    bt = [torch.from_numpy(b[k]).to(dev) for k in range(NRHS)]
    xt = [torch.zeros_like(t) for t in bt]
    g = H.hisq_gauge_load(L1, dU, dN, prec=H.HISQ_F32, recon_U=18, recon_N=14)
    t, st = _time_solve(H, torch, g, MASS1, 0.0, bt, xt, TOL,
                        H.cg_params(inner_prec=H.HISQ_F32, reliable_every=RELIABLE_EVERY1), stream)
    H.hisq_gauge_free(g)
    g = H.hisq_gauge_load(L1, dU, dN, prec=H.HISQ_F64)
    x64 = [torch.zeros_like(bt[0])]
    t64, st64 = _time_solve(H, torch, g, MASS1, 0.0, bt[:1], x64, TOL, H.cg_params(inner_prec=H.HISQ_F64),
                            stream)
    H.hisq_gauge_free(g)
    return {"workload": "HISQ even-odd CG, 32^3x8, n=8 Z2 rhs, m=0.01, FP32 storage (U r18, N r14), "
                        "FP64 reliable updates every 50, tol 1e-10",
            "s_per_rhs": t / NRHS, "iterations": st.total_iters, "reliable_updates": st.reliable_updates,
            "max_true_rel_res": max(st.true_rel_res[k] for k in range(NRHS)),
            "fp64_single_rhs_s": t64, "fp64_iterations": st64.total_iters,
            "mixed_over_fp64_time": (t / NRHS) / t64}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def _oracle_cg_iteration_seconds(apply_A, b, iters: int) -> float:
    from oracle import hisq_oracle as O
    t0 = time.perf_counter()
    O.cg(apply_A, b, tol=1e-300, maxiter=iters)
    return (time.perf_counter() - t0) / iters


_WORKER = {}


def _oracle_worker_init(Ls):
    """Links and sources of the all-core sample, built once per spawned process."""
    import hisq_inputs as gen
    _WORKER["L"] = Ls
    _WORKER["links"] = gen.hisq_links(Ls, seed=LINK_SEED)
    _WORKER["b"] = gen.z2_source(Ls, NRHS, seed=SOURCE_SEED)


def _oracle_sample_worker(job):
    """CG iterations of one rhs of the all-core sample (in a spawned process)."""
    from oracle import hisq_oracle as O
    mass, k, iters = job
    U, N = _WORKER["links"]
    Ls = _WORKER["L"]
    t0 = time.perf_counter()
    O.cg(lambda q: O.apply_Ae(U, N, q, Ls, mass), _WORKER["b"][k:k + 1], tol=1e-300, maxiter=iters)
    return time.perf_counter() - t0


def run_oracle_timing(args):
    """The FP64 oracle on the host cores for every configuration: one Dslash
    call, and CG seconds per rhs (to convergence on 8^4; elsewhere a bounded
    sample of iterations scaled by the iteration count of that system). The
    all-core line runs the 8 rhs of the 32^3x8 bundle as 8 spawned processes."""
    import multiprocessing as mp

    import hisq_inputs as gen
    from oracle import hisq_oracle as O
    cpus = os.cpu_count() or 1

    def line(d):
        d.update({"impl": "reference", "kind": "oracle", "host_cpus": cpus})
        print(json.dumps(d), flush=True)

    def dslash_s(U, N, v, Ls):
        t0 = time.perf_counter()
        O.dslash_parity(U, N, v, Ls, 0)
        return time.perf_counter() - t0

    # 8^4, FP64, one rhs, m = 0.05, to convergence
    L0 = (8, 8, 8, 8)
    U, N = gen.hisq_links(L0, seed=0)
    b = gen.z2_source(L0, 1, seed=0)
    t0 = time.perf_counter()
    _, it = O.cg(lambda q: O.apply_Ae(U, N, q, L0, 0.05), b, tol=TOL)
    line({"workload": "oracle 8^4 m=0.05", "cores": 1, "cg_s_per_rhs": time.perf_counter() - t0,
          "cg_iterations": int(it[0]), "dslash_s_per_call_1rhs": dslash_s(U, N, b, L0),
          "sample": "complete solve"})

    # 32^3x8, m = 0.01
    U, N = gen.hisq_links(L1, seed=LINK_SEED)
    b = gen.z2_source(L1, NRHS, seed=SOURCE_SEED)
    iters_total, how = fp64_iterations(None)
    t_it = _oracle_cg_iteration_seconds(lambda q: O.apply_Ae(U, N, q, L1, MASS1), b[:1], 2)
    line({"workload": "oracle 32^3x8 m=0.01", "cores": 1, "cg_s_per_rhs": t_it * iters_total,
          "cg_iterations": iters_total, "iterations_from": how,
          "dslash_s_per_call_8rhs": dslash_s(U, N, b, L1),
          "sample": f"2 CG iterations of one rhs ({t_it:.3f} s/iteration)"})
    procs = min(NRHS, cpus)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_oracle_worker_init, initargs=(L1,)) as pool:
        pool.map(_oracle_sample_worker, [(MASS1, 0, 1)] * procs, chunksize=1)     # warm-up
        t0 = time.perf_counter()
        pool.map(_oracle_sample_worker, [(MASS1, k, 2) for k in range(NRHS)], chunksize=1)
        wall = time.perf_counter() - t0
    per_it_bundle = wall / 2
    line({"workload": "oracle 32^3x8 m=0.01, all cores", "cores": procs,
          "cg_s_per_rhs": per_it_bundle * iters_total / NRHS, "cg_iterations": iters_total,
          "sample": f"2 CG iterations of each of the {NRHS} rhs in {procs} spawned processes"})
    del U, N, b

    # 48^3x12, m = 0.0025, Gaussian; iteration count of the GPU FP64 solve
    L2 = (48, 48, 48, 12)
    U, N = gen.hisq_links(L2, seed=LINK_SEED)
    b = gen.gaussian_source(L2, 1, seed=SOURCE_SEED)
    t_it = _oracle_cg_iteration_seconds(lambda q: O.apply_Ae(U, N, q, L2, 0.0025), b, 1)
    line({"workload": "oracle 48^3x12 m=0.0025", "cores": 1, "cg_s_per_rhs": t_it * 11310,
          "cg_iterations": 11310, "iterations_from": "FP64 GPU solve of the same system",
          "dslash_s_per_call_1rhs": dslash_s(U, N, b, L2),
          "sample": f"1 CG iteration of one rhs ({t_it:.2f} s/iteration)"})
    del U, N, b

    # 16^4, mu = 0.1, full lattice M^dag M, m = 0.05
    L3 = (16, 16, 16, 16)
    U, N = gen.hisq_links(L3, seed=LINK_SEED)
    v = O.to_full(gen.z2_source(L3, 1, seed=SOURCE_SEED), L3, 0) + \
        O.to_full(gen.z2_source(L3, 1, seed=SOURCE_SEED + 7), L3, 1)
    t_it = _oracle_cg_iteration_seconds(lambda q: O.apply_MdagM(U, N, q, 0.05, 0.1), v, 2)
    line({"workload": "oracle 16^4 mu=0.1 full lattice", "cores": 1, "cg_s_per_rhs": t_it * 930,
          "cg_iterations": 930, "iterations_from": "FP64 GPU solve of the same system",
          "sample": f"2 CG iterations of one rhs ({t_it:.3f} s/iteration)"})


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "oracle-timing":
        run_oracle_timing(args)
        return
    import hisq_inputs as gen
    U, N = gen.hisq_links(L, seed=LINK_SEED)
    b = gen.gaussian_source(L, NRHS, seed=SOURCE_SEED)
    iters_total, how = fp64_iterations(11310, mixed=True)
    if how.startswith("iteration count of the FP64 GPU"):
        how = "iteration count of the FP64 GPU solve of the same system, measured separately"
    per_step_iters = 1
    for _ in range(args.warmup):
        oracle_sample(U, N, b[:1], per_step_iters)
    ts = [oracle_sample(U, N, b[:1], per_step_iters) for _ in range(args.steps)]
    t_it = sum(ts) / len(ts)
    value = t_it * iters_total if iters_total else None
    sample = (f"{per_step_iters} numpy FP64 oracle CG iteration per step, 1 rhs on 48^3x12 "
              f"({t_it:.3f} s/iteration), scaled by {iters_total} iterations ({how})")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_it * per_step_iters * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Haar-random links, Gaussian sources; seeded)", "config": workload_config(world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# further workloads (besides the headline JSON line): --workload <name>
# ---------------------------------------------------------------------------

def _time_solve(H, torch, g, mass, mu, bt, xt, tol, params, stream, reps=1):
    """CUDA-event seconds of one hisq_cg_solve (after one warm-up) and its stats."""
    st = H.hisq_cg_solve(g, mass, mu, bt, xt, tol, params, stream=stream)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = H.hisq_cg_solve(g, mass, mu, bt, xt, tol, params, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(ts), st


def _cg_line(name, lattice, n, inner, t, st, extra=None):
    d = {"workload": name, "lattice": list(lattice), "nrhs": n, "inner_prec": inner,
         "s_per_solve": t, "s_per_rhs": t / n, "iterations": st.total_iters,
         "reliable_updates": st.reliable_updates,
         "max_true_rel_res": max(st.true_rel_res[k] for k in range(n))}
    if extra:
        d.update(extra)
    print(json.dumps(d), flush=True)


def run_cg_configs(args):
    """CG seconds per rhs on the listed configurations: FP64 8^4 single rhs;
    FP32 32^3x8 with n = 1, 2, 4, 8 (and the FP64 single-rhs solve); FP16
    48^3x12 with n = 8 Gaussian sources at m = 0.0025 against the FP64
    single-rhs solve of source 0; FP64 16^4 full-lattice solve at mu = 0.1."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    H.hisq.library()

    def dev_list(a):
        return [torch.from_numpy(np.ascontiguousarray(a[k])).to(dev) for k in range(a.shape[0])]

    # 8^4, FP64, one rhs, seed 0, m = 0.05
    L0 = (8, 8, 8, 8)
    U, N = gen.hisq_links(L0, seed=0)
    g = H.hisq_gauge_load(L0, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev), prec=H.HISQ_F64)
    bt = dev_list(gen.z2_source(L0, 1, seed=0))
    xt = [torch.zeros_like(bt[0])]
    t, st = _time_solve(H, torch, g, 0.05, 0.0, bt, xt, TOL, H.cg_params(inner_prec=H.HISQ_F64), stream, 3)
    _cg_line("fp64 8^4 m=0.05", L0, 1, "f64", t, st)
    H.hisq_gauge_free(g)

    # 32^3x8, FP32 inner, n = 1, 2, 4, 8, and FP64 single rhs
    U, N = gen.hisq_links(L1, seed=LINK_SEED)
    dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
    b = gen.z2_source(L1, NRHS, seed=SOURCE_SEED)
    g = H.hisq_gauge_load(L1, dU, dN, prec=H.HISQ_F32, recon_U=18, recon_N=14)
    for n in (1, 2, 4, 8):
        bt = dev_list(b[:n])
        xt = [torch.zeros_like(x) for x in bt]
        t, st = _time_solve(H, torch, g, MASS1, 0.0, bt, xt, TOL,
                            H.cg_params(inner_prec=H.HISQ_F32, reliable_every=RELIABLE_EVERY1), stream)
        _cg_line("fp32 32^3x8 m=0.01", L1, n, "f32", t, st)
    H.hisq_gauge_free(g)
    g = H.hisq_gauge_load(L1, dU, dN, prec=H.HISQ_F64)
    bt = dev_list(b[:1])
    xt = [torch.zeros_like(bt[0])]
    t, st = _time_solve(H, torch, g, MASS1, 0.0, bt, xt, TOL, H.cg_params(inner_prec=H.HISQ_F64), stream)
    _cg_line("fp64 32^3x8 m=0.01", L1, 1, "f64", t, st)
    H.hisq_gauge_free(g)
    del dU, dN

    # 48^3x12, FP16 storage / FP32 arithmetic, n = 8 Gaussian, m = 0.0025; FP64 single rhs
    L2 = (48, 48, 48, 12)
    U, N = gen.hisq_links(L2, seed=LINK_SEED)
    dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
    del U, N
    b = gen.gaussian_source(L2, 8, seed=SOURCE_SEED)
    g = H.hisq_gauge_load(L2, dU, dN, prec=H.HISQ_F16, recon_U=18, recon_N=14)
    bt = dev_list(b)
    xt = [torch.zeros_like(x) for x in bt]
    t16, st16 = _time_solve(H, torch, g, 0.0025, 0.0, bt, xt, TOL,
                            H.cg_params(inner_prec=H.HISQ_F16, reliable_every=RELIABLE_EVERY), stream)
    H.hisq_gauge_free(g)
    g = H.hisq_gauge_load(L2, dU, dN, prec=H.HISQ_F64)
    x64 = [torch.zeros_like(bt[0])]
    t64, st64 = _time_solve(H, torch, g, 0.0025, 0.0, bt[:1], x64, TOL, H.cg_params(inner_prec=H.HISQ_F64), stream)
    diff = float(torch.linalg.vector_norm(xt[0] - x64[0]) / torch.linalg.vector_norm(x64[0]))
    _cg_line("fp16 48^3x12 m=0.0025 gaussian", L2, 8, "f16", t16, st16,
             {"fp64_single_rhs_s": t64, "fp64_iterations": st64.total_iters,
              "mixed_over_fp64_s_per_rhs": (t16 / 8) / t64, "rhs0_rel_diff_vs_fp64": diff})
    H.hisq_gauge_free(g)
    del dU, dN

    # 16^4, FP64, n = 4 Z2, mu = 0.1, full-lattice M^dag M, m = 0.05
    L3 = (16, 16, 16, 16)
    U, N = gen.hisq_links(L3, seed=LINK_SEED)
    g = H.hisq_gauge_load(L3, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev), prec=H.HISQ_F64)
    vh = int(np.prod(L3)) // 2
    bz = gen.z2_source(L3, 4, seed=SOURCE_SEED)
    bfull = np.concatenate([bz, gen.z2_source(L3, 4, seed=SOURCE_SEED + 7)], axis=1)
    assert bfull.shape[1] == 2 * vh
    bt = dev_list(bfull)
    xt = [torch.zeros_like(x) for x in bt]
    t, st = _time_solve(H, torch, g, 0.05, 0.1, bt, xt, TOL,
                        H.cg_params(inner_prec=H.HISQ_F64, even_odd=0), stream)
    _cg_line("fp64 16^4 mu=0.1 full lattice", L3, 4, "f64", t, st)
    H.hisq_gauge_free(g)


def run_dslash_sweep(args):
    """Autotuned Dslash (AoS spinors) for n = 1..16 on 48^3x12 and 64^3x16 in
    FP64 18/18, FP32 18/14, FP16 18/14 and FP16 12/14, and on the bundle
    layout for n = 4, 8, 16: time per launch, algorithmic GB/s and its
    fraction of the measured HBM peak, GFlop/s."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    H.hisq.library()
    peak = measured_peaks()
    sizes = {H.HISQ_F64: 8, H.HISQ_F32: 4, H.HISQ_F16: 2}
    names = {H.HISQ_F64: "f64", H.HISQ_F32: "f32", H.HISQ_F16: "f16"}
    dtypes = {H.HISQ_F64: torch.complex128, H.HISQ_F32: torch.complex64, H.HISQ_F16: torch.float16}
    lattices = [tuple(int(x) for x in s.split("x")) for s in args.lattices.split(",")]
    for Ls in lattices:
        U, N = gen.hisq_links(Ls, seed=LINK_SEED)
        dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
        del U, N
        vh = int(np.prod(Ls)) // 2
        for prec, ru, rn in ((H.HISQ_F64, 18, 18), (H.HISQ_F32, 18, 14), (H.HISQ_F16, 18, 14),
                             (H.HISQ_F16, 12, 14)):
            g = H.hisq_gauge_load(Ls, dU, dN, prec=prec, recon_U=ru, recon_N=rn)
            for n in (1, 2, 4, 8, 16):
                shape = (vh, 3, 2) if prec == H.HISQ_F16 else (vh, 3)
                vs = [torch.randn(shape, dtype=torch.float32, device=dev).to(dtypes[prec]) if prec == H.HISQ_F16
                      else torch.randn(shape, dtype=dtypes[prec], device=dev) for _ in range(n)]
                ws = [torch.empty_like(v) for v in vs]
                tune = H.hisq_autotune_dslash(g, n, prec, H.HISQ_AOS, 5)
                for _ in range(3):
                    H.hisq_dslash(g, vs, ws, 0, prec, stream=stream)
                reps = 20
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps):
                    H.hisq_dslash(g, vs, ws, 0, prec, stream=stream)
                e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1) / 1e3 / reps
                nb = dslash_bytes_per_site(n, ru, rn, sizes[prec], sizes[prec]) * vh
                print(json.dumps({"workload": "dslash sweep", "lattice": list(Ls), "prec": names[prec],
                                  "recon": [ru, rn], "n": n, "us": round(t * 1e6, 2),
                                  "alg_gbs": round(nb / t / 1e9, 1),
                                  "frac_of_measured_hbm": round(nb / t / 1e9 / peak["hbm_gbs"], 4),
                                  "gflops": round(DSLASH_FLOPS_PER_SITE_RHS * n * vh / t / 1e9, 1),
                                  "mapping": [tune["rhs_per_thread"], tune["min_blocks"], tune["flags"]]}),
                      flush=True)
                del vs, ws
            if prec != H.HISQ_F64:
                # the CG's own layout: rhs-interleaved bundle chunks
                for n in (4, 8, 16):
                    src = [torch.randn(vh, 3, dtype=torch.complex128, device=dev) for _ in range(n)]
                    el = 4 if prec == H.HISQ_F32 else 2
                    vb = torch.empty(H.hisq.bundle_bytes(g, n, prec) // el,
                                     dtype=torch.float32 if prec == H.HISQ_F32 else torch.float16, device=dev)
                    H.hisq_bundle_pack(g, src, prec, vb)
                    wb = torch.empty_like(vb)
                    del src
                    tune = H.hisq_autotune_dslash(g, n, prec, H.HISQ_BUNDLE, 5)
                    for _ in range(3):
                        H.hisq_dslash_ex(g, 0.0, vb, wb, 0, prec, H.HISQ_BUNDLE, stream=stream, n=n)
                    reps = 20
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(reps):
                        H.hisq_dslash_ex(g, 0.0, vb, wb, 0, prec, H.HISQ_BUNDLE, stream=stream, n=n)
                    e1.record(stream)
                    e1.synchronize()
                    t = e0.elapsed_time(e1) / 1e3 / reps
                    nb = dslash_bytes_per_site(n, ru, rn, sizes[prec], sizes[prec]) * vh
                    print(json.dumps({"workload": "dslash sweep", "layout": "bundle", "lattice": list(Ls),
                                      "prec": names[prec], "recon": [ru, rn], "n": n, "us": round(t * 1e6, 2),
                                      "alg_gbs": round(nb / t / 1e9, 1),
                                      "frac_of_measured_hbm": round(nb / t / 1e9 / peak["hbm_gbs"], 4),
                                      "gflops": round(DSLASH_FLOPS_PER_SITE_RHS * n * vh / t / 1e9, 1),
                                      "mapping": [tune["rhs_per_thread"], tune["min_blocks"], tune["flags"]]}),
                          flush=True)
                    del vb, wb
            H.hisq_gauge_free(g)
        del dU, dN
        torch.cuda.empty_cache()


def run_batched(args):
    """Three gauge fields of uneven volume solved by one hisq_cg_solve_batched
    call (one CUDA graph holding a device-driven loop per problem): 24^3x6 with n = 16
    (m = 0.002), 32^3x8 with n = 8 (m = 0.01), 64^3x16 with n = 4 (m = 0.01);
    FP16 storage with FP32 arithmetic and FP64 reliable updates, Z2 sources,
    link compression and thread mapping chosen by the autotuner. Also times
    the same three solves one after another."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    H.hisq.library()
    cases = [((24, 24, 24, 6), 16, 0.002), ((32, 32, 32, 8), 8, 0.01), ((64, 64, 64, 16), 4, 0.01)]
    handles, probs, tuned = [], [], []
    for i, (Ls, n, m) in enumerate(cases):
        U, N = gen.hisq_links(Ls, seed=LINK_SEED)
        dU, dN = torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev)
        del U, N
        g = H.hisq_gauge_load_tuned(Ls, dU, dN, prec=H.HISQ_F16, n=n)
        del dU, dN
        handles.append(g)
        bundle = H.hisq_autotune_bundle(g, n, H.HISQ_F16)
        tuned.append({"lattice": list(Ls), "n": n, "mass": m, "recon": [g.recon_U, g.recon_N],
                      "mapping": list(H.hisq_get_dslash_mapping_ex(g, n, H.HISQ_F16, H.HISQ_BUNDLE)),
                      "bundle_tuner_best_n": bundle["n"]})
        b = gen.z2_source(Ls, n, seed=SOURCE_SEED + i)
        bt = [torch.from_numpy(b[k]).to(dev) for k in range(n)]
        probs.append(dict(g=g, mass=m, mu=0.0, b=bt, x=[torch.zeros_like(t) for t in bt], tol=TOL))
        torch.cuda.empty_cache()
    params = H.cg_params(inner_prec=H.HISQ_F16, reliable_every=RELIABLE_EVERY1)
    H.hisq_cg_solve_batched(probs, params, stream=stream)        # warm-up (graphs, workspaces)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = H.hisq_cg_solve_batched(probs, params, stream=stream)
    e1.record(stream)
    e1.synchronize()
    t_batched = e0.elapsed_time(e1) / 1e3
    alone = []
    for pr in probs:      # each problem alone, one after another
        e0.record(stream)
        H.hisq_cg_solve(pr["g"], pr["mass"], 0.0, pr["b"], pr["x"], TOL, params, stream=stream)
        e1.record(stream)
        e1.synchronize()
        alone.append(e0.elapsed_time(e1) / 1e3)
    t_seq = sum(alone)
    # the two smaller problems batched without the largest: do they overlap
    # each other where the largest leaves no room?
    small = sorted(range(len(probs)), key=lambda i: alone[i])[:2]
    e0.record(stream)
    H.hisq_cg_solve_batched([probs[i] for i in small], params, stream=stream)
    e1.record(stream)
    e1.synchronize()
    t_small_pair = e0.elapsed_time(e1) / 1e3
    nrhs = sum(n for _, n, _ in cases)
    for tinfo, st, (Ls, n, m), ta in zip(tuned, stats, cases, alone):
        tinfo.update({"iterations": st.total_iters, "reliable_updates": st.reliable_updates,
                      "max_true_rel_res": max(st.true_rel_res[k] for k in range(n)), "s_alone": ta})
    print(json.dumps({"workload": "batched uneven lattices, FP16 inner", "s_batched": t_batched,
                      "s_sequential": t_seq, "s_longest_alone": max(alone),
                      "batched_over_longest_alone": t_batched / max(alone),
                      "s_batched_two_smaller": t_small_pair,
                      "s_two_smaller_alone": [alone[i] for i in small],
                      "s_per_rhs_batched": t_batched / nrhs, "nrhs": nrhs, "problems": tuned}), flush=True)
    for g in handles:
        H.hisq_gauge_free(g)


def run_inverter_sweep(args):
    """Inverter GFlop/s with 4 rhs against lattice size (the paper's Fig. 4,
    right): 300 CG iterations of the FP32-inner even-odd solve at m = 0.01
    on each lattice, flops 2 x 1146 + 12 (mass term) + 60 (vector updates) per
    even site, rhs and iteration, reliable updates included in the time."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    H.hisq.library()
    n, iters = 4, 300
    for Ls in ((16, 16, 16, 16), (24, 24, 24, 6), (32, 32, 32, 8), (48, 48, 48, 12), (64, 64, 64, 16)):
        U, N = gen.hisq_links(Ls, seed=LINK_SEED)
        g = H.hisq_gauge_load(Ls, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev),
                              prec=H.HISQ_F32, recon_U=18, recon_N=14)
        del U, N
        b = gen.z2_source(Ls, n, seed=SOURCE_SEED)
        bt = [torch.from_numpy(b[k]).to(dev) for k in range(n)]
        xt = [torch.zeros_like(t) for t in bt]
        p = H.cg_params(inner_prec=H.HISQ_F32, reliable_every=RELIABLE_EVERY1, maxiter=iters)

        def solve():
            try:
                return H.hisq_cg_solve(g, MASS1, 0.0, bt, xt, 1e-30, p, stream=stream)
            except H.HisqError as e:          # HISQ_ENOCONV at maxiter: stats ride on the error
                return e.stats
        solve()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = solve()
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        vh = int(np.prod(Ls)) // 2
        flops = (2 * DSLASH_FLOPS_PER_SITE_RHS + 12 + 60) * vh * n * st.total_iters
        print(json.dumps({"workload": "inverter sweep, n=4, FP32 inner", "lattice": list(Ls),
                          "iterations": st.total_iters, "reliable_updates": st.reliable_updates,
                          "s": t, "gflops": round(flops / t / 1e9, 1),
                          "us_per_iteration": round(t / st.total_iters * 1e6, 1)}), flush=True)
        H.hisq_gauge_free(g)
        del bt, xt
        torch.cuda.empty_cache()


def run_dslash_probe(args):
    """A fixed number of Dslash (or normal-operator) launches of one kernel
    configuration, for ncu captures and event timing outside the headline:
    prints one JSON line with the CUDA-event time per launch, the algorithmic
    GB/s (8 (f_U + f_N) s_l + 12 n s_s bytes per output site) and GFlop/s."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H

    precs = {"f64": H.HISQ_F64, "f32": H.HISQ_F32, "f16": H.HISQ_F16}
    sbytes = {"f64": 8, "f32": 4, "f16": 2}
    Ls = tuple(args.lattice)
    prec = precs[args.prec]
    n = args.n
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    H.hisq.library()
    U, N = gen.hisq_links(Ls, seed=LINK_SEED)
    fu, fn = (18, 18) if prec == H.HISQ_F64 else tuple(args.recon)
    g = H.hisq_gauge_load(Ls, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev), prec=prec,
                          recon_U=fu, recon_N=fn)
    del U, N
    if args.rpt or args.minb or args.flags:
        H.hisq_set_dslash_mapping(g, args.rpt, args.minb, args.flags)
    layout = {"aos": H.HISQ_AOS, "soa": H.HISQ_SOA, "bundle": H.HISQ_BUNDLE}[args.layout]
    vh = int(np.prod(Ls)) // 2
    stream = torch.cuda.current_stream(dev)
    if layout == H.HISQ_BUNDLE:
        src = [torch.randn(vh, 3, dtype=torch.complex128, device=dev) for _ in range(n)]
        dt = torch.float32 if prec == H.HISQ_F32 else torch.float16
        vb = torch.empty(H.hisq.bundle_bytes(g, n, prec) // (4 if prec == H.HISQ_F32 else 2), dtype=dt,
                         device=dev)
        H.hisq_bundle_pack(g, src, prec, vb)
        wb = torch.empty_like(vb)
        del src
    else:
        if prec == H.HISQ_F64:
            vs = [torch.randn(vh, 3, dtype=torch.complex128, device=dev) for _ in range(n)]
        elif prec == H.HISQ_F32:
            vs = [torch.randn(vh, 3, dtype=torch.complex64, device=dev) for _ in range(n)]
        else:
            vs = [torch.randn(vh, 3, 2, device=dev).half() for _ in range(n)]
        ws = [torch.empty_like(v) for v in vs]

    def launch():
        if args.op == "mdagm":
            H.hisq_mdagm(g, 0.01, vs, ws, prec, stream=stream)
        elif layout == H.HISQ_BUNDLE:
            H.hisq_dslash_ex(g, args.mu, vb, wb, 0, prec, layout, stream=stream, n=n)
        else:
            H.hisq_dslash_ex(g, args.mu, vs, ws, 0, prec, layout, stream=stream)

    for _ in range(args.warmup):
        launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        launch()
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.reps
    ops = 2 if args.op == "mdagm" else 1
    nb = dslash_bytes_per_site(n, fu, fn, sbytes[args.prec], sbytes[args.prec]) * vh
    print(json.dumps({"workload": "dslash probe", "lattice": list(Ls), "n": n, "prec": args.prec,
                      "recon": [fu, fn], "op": args.op, "layout": args.layout, "rpt": args.rpt,
                      "minb": args.minb, "flags": args.flags, "us_per_launch": t * 1e6 / ops,
                      "alg_bytes_per_dslash": nb, "alg_gbs": nb * ops / t / 1e9,
                      "gflops": DSLASH_FLOPS_PER_SITE_RHS * n * vh * ops / t / 1e9}), flush=True)
    H.hisq_gauge_free(g)


def run_cg_probe(args):
    """One solve of the headline system (48^3x12, n = 8, m = 0.0025; FP16
    storage, or --prec f32 / f64) capped at --maxiter iterations, for launch
    lists, captures of the solve's kernels and storage comparisons; prints
    iterations and seconds."""
    import torch

    import hisq_inputs as gen
    import paper_1411_4439_gb300 as H
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    H.hisq.library()
    Ls = tuple(args.lattice)
    U, N = gen.hisq_links(Ls, seed=LINK_SEED)
    prec = {"f16": H.HISQ_F16, "f32": H.HISQ_F32, "f64": H.HISQ_F64}[args.prec]
    g = H.hisq_gauge_load(Ls, torch.from_numpy(U).to(dev), torch.from_numpy(N).to(dev), prec=prec,
                          recon_U=18 if prec == H.HISQ_F64 else args.recon[0],
                          recon_N=18 if prec == H.HISQ_F64 else args.recon[1])
    del U, N
    b = gen.gaussian_source(Ls, args.n, seed=SOURCE_SEED)
    bt = [torch.from_numpy(b[k]).to(dev) for k in range(args.n)]
    xt = [torch.zeros_like(t) for t in bt]
    p = H.cg_params(inner_prec=prec, reliable_every=args.reliable_every or RELIABLE_EVERY,
                    maxiter=args.maxiter, device_loop=args.device_loop)
    for _ in range(2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            st = H.hisq_cg_solve(g, MASS, 0.0, bt, xt, TOL, p, stream=stream)
        except H.HisqError as e:      # HISQ_ENOCONV at the cap: the stats ride on the error
            st = e.stats
        torch.cuda.synchronize()
        print(json.dumps({"workload": "cg probe", "lattice": list(Ls), "n": args.n, "prec": args.prec,
                          "reliable_every": p.reliable_every, "iterations": st.total_iters,
                          "reliable_updates": st.reliable_updates,
                          "max_true_rel_res": max(st.true_rel_res[k] for k in range(args.n)),
                          "s": time.perf_counter() - t0}), flush=True)
    H.hisq_gauge_free(g)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["headline", "cg-configs", "dslash-sweep", "batched", "inverter-sweep",
                                           "oracle-timing", "dslash-probe", "cg-probe"],
                    default="headline",
                    help="headline = the one JSON line of the contract; oracle-timing needs --impl reference")
    ap.add_argument("--lattices", default="48x48x48x12,64x64x64x16",
                    help="lattices of the Dslash sweep (Lx x Ly x Lz x Lt, comma separated)")
    # dslash-probe: one kernel configuration
    ap.add_argument("--lattice", type=int, nargs=4, default=[48, 48, 48, 12])
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--prec", choices=["f64", "f32", "f16"], default="f16")
    ap.add_argument("--recon", type=int, nargs=2, default=[18, 14])
    ap.add_argument("--layout", choices=["aos", "soa", "bundle"], default="bundle")
    ap.add_argument("--rpt", type=int, default=0)
    ap.add_argument("--minb", type=int, default=0)
    ap.add_argument("--flags", type=int, default=0, help="HISQ_MAP_* bits")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--mu", type=float, default=0.0)
    ap.add_argument("--op", choices=["dslash", "mdagm"], default="dslash")
    ap.add_argument("--maxiter", type=int, default=400, help="cg-probe: iteration cap")
    ap.add_argument("--reliable-every", type=int, default=0,
                    help="cg-probe: FP64 reliable update every K iterations (0: the headline's)")
    ap.add_argument("--device-loop", type=int, choices=[0, 1], default=1,
                    help="cg-probe: 1 = the whole solve as one graph launch, 0 = one launch per kernel")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cg-configs":
        run_cg_configs(args)
    elif args.workload == "dslash-sweep":
        run_dslash_sweep(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "inverter-sweep":
        run_inverter_sweep(args)
    elif args.workload == "dslash-probe":
        run_dslash_probe(args)
    elif args.workload == "cg-probe":
        run_cg_probe(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
