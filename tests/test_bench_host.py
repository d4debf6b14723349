"""Host-side logic of bench.py: byte accounting and the multi-rank timing reduction.

The multi-GPU path shards independent rhs bundles across ranks (weak
scaling, no data-path collective); the only collectives are a barrier and
the max-over-ranks of the step time. They run here as two gloo ranks on CPU.
"""
import os
import socket

import pytest

import bench
from oracle import hisq_oracle as O


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("fu,fn,sl,ss", [(18, 18, 8, 8), (18, 14, 4, 4), (18, 14, 2, 2), (12, 14, 2, 2)])
def test_algorithmic_bytes_match_oracle_model(n, fu, fn, sl, ss):
    assert bench.dslash_bytes_per_site(n, fu, fn, sl, ss) == O.dslash_bytes_algorithmic(n, fu, fn, sl, ss)


def test_byte_table_values():
    # bytes per output site: FP32 18/14 at n = 8 is 1408, FP16 12/14 at n = 1 is 440
    assert bench.dslash_bytes_per_site(8, 18, 14, 4, 4) == 1408
    assert bench.dslash_bytes_per_site(1, 12, 14, 2, 2) == 440
    assert bench.dslash_bytes_per_site(16, 18, 18, 8, 8) == 3840


def test_rank_bundles_are_distinct():
    seeds = {bench.source_seed_for_rank(r) for r in range(8)}
    assert len(seeds) == 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t = bench.reduce_max(1.0 + rank, world)
        q.put((rank, t))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_rank_max_reduction_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    assert got == {0: 2.0, 1: 2.0}


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    """Under torchrun only rank 0 runs and prints the reference line."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.main(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert capsys.readouterr().out == ""


def test_fp32_peak_and_roofline_bound():
    # 152 SMs x 128 lanes x 2 flop x 2070 MHz
    assert bench.fp32_peak_tflops(152, 2070.0) == pytest.approx(80.548, abs=1e-3)
    peak, hbm = bench.fp32_peak_tflops(152, 2070.0), 6777.0
    vh = 663552
    f16 = (bench.DSLASH_FLOPS_PER_SITE_RHS * 8 * vh, bench.dslash_bytes_per_site(8, 18, 14, 2, 2) * vh)
    f32 = (bench.DSLASH_FLOPS_PER_SITE_RHS * 8 * vh, bench.dslash_bytes_per_site(8, 18, 14, 4, 4) * vh)
    assert bench.roofline_bound(*f16, peak, hbm) == "alu"     # 13.0 flop/B past the ridge of 11.9
    assert bench.roofline_bound(*f32, peak, hbm) == "hbm"     # 6.5 flop/B


def test_roofline_traffic_only_for_a_captured_configuration():
    assert bench.dslash_traffic("f16", (48, 48, 48, 12), 8, (3, 3, 3)) is None
    for key, value in bench.DSLASH_TRAFFIC.items():
        assert bench.dslash_traffic(key[0], key[1], key[2], key[3:]) == value > 0


def test_warmup_is_clamped_to_three():
    seen = {}

    def fake(args):
        seen["warmup"] = args.warmup
    old = bench.run_reference
    bench.run_reference = fake
    try:
        bench.main(["--impl", "reference", "--warmup", "1"])
    finally:
        bench.run_reference = old
    assert seen["warmup"] == 3


def test_cg_kernel_byte_minima_follow_the_dslash_byte_model():
    """The first Dslash of an iteration moves the algorithmic bytes of one
    Dslash; the second also reads p for its epilogue; the vector updates move
    three (r) and three plus two FP32 (x/p) vectors of the bundle."""
    from oracle import hisq_oracle as O
    vh, n = 663552, 8
    m = bench.cg_kernel_byte_minima(vh, n)
    assert m["dslash_t"] == O.dslash_bytes_algorithmic(n, 18, 14, 2, 2) * vh == 467140608
    assert m["dslash_ap_alpha"] - m["dslash_t"] == 6 * 2 * n * vh
    assert m["update_r"] == 191102976
    assert m["update_px"] == 445906944
