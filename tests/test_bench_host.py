"""Host-side logic of bench.py on CPU: the multi-rank timing helpers over a
world of two gloo ranks, and the clock-record parser."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    t = bench.max_over_ranks(world, 1.5 + rank)   # rank 1 is the slow one
    bench.barrier(world)
    q.put((rank, t))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 2.5, 1: 2.5}


def test_single_rank_helpers_are_identity():
    bench.barrier(1)
    assert bench.max_over_ranks(1, 3.25) == 3.25


def test_clock_parser():
    text = "\n".join([
        "0, 1980, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2010, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ])
    rec = bench.ClockSampler.parse(text)
    assert rec["sm_mhz"] == 2010 and rec["sm_max_mhz"] == 2070 and rec["samples"] == 3
    assert rec["reasons"] == ["sw_power_cap"]
    assert bench.ClockSampler.parse("") is None


def test_roofline_instruction_counts_follow_the_rotation_forms():
    """Per site-update: 16 collision and 2 potential rotations per live pair
    (1 pair in E_z mode, 2 with six planes).  FP32 collisions take 8
    instructions (two-word coefficients), potential rotations 6; FP64
    collisions 3 (three shears), potential rotations 4; double-single rows 23
    per output.  3D: per axis 16 collision rotations on 2 pairs, then six
    potential rotations."""
    assert bench.alu_ops_per_su(3, 4) == 16 * 8 + 2 * 6
    assert bench.alu_ops_per_su(6, 4) == 2 * (16 * 8 + 2 * 6)
    assert bench.alu_ops_per_su(3, 8) == 16 * 3 + 2 * 4
    assert bench.alu_ops_per_su(6, 8) == 2 * (16 * 3 + 2 * 4)
    assert bench.ds_ops_per_su(3) == 18 * 2 * 23
    assert bench.alu_ops_per_su_3d(4) == 3 * 16 * 8 + 6 * 6
    assert bench.alu_ops_per_su_3d(8) == 3 * 16 * 3 + 6 * 4
    bench.DEVICE.update(sms=152, sm_max_mhz=2070.0)
    r = bench.roofline(3, 8, 8.6e9, None)
    assert r["bound"] == "alu" and r["ops_per_site_update"] == 56
    assert r["frac"] == pytest.approx(8.6e9 * 56 / (bench.FP64_NOMINAL_FLOPS / 2))
    assert r["peak_kind"].startswith("nominal")
    assert bench.fp32_inst_peak() == pytest.approx(152 * 128 * 2.07e9)
    r = bench.roofline(3, 4, 1.26e11, None)
    assert r["bound"] == "hbm" and r["bytes_per_site_update"] == 24


def test_cpu_model_is_named():
    m = bench.cpu_model()
    assert isinstance(m, str) and m.strip()
