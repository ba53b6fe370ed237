"""Host-side logic of bench.py without a GPU: argument defaults, the clock
summary, and the max-over-ranks timing of the N > 1 path on two gloo ranks."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_defaults():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.steps >= 1 and a.impl == "gb300" and a.mode == "both"


def test_clock_summary_parses_nvidia_smi_csv(tmp_path):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "c.csv")
    with open(c.path, "w") as fh:
        fh.write("0, 1900, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        fh.write("0, 1950, 2070, 1001.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        fh.write("0, 1920, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    s = c.summary()
    assert s["sm_mhz"] == 1920 and s["sm_max_mhz"] == 2070 and s["reasons"] == ["sw_power_cap"]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.reduce_max(10.0 + rank, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, got))


def test_reduce_max_over_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 11.0), (1, 11.0)]


def test_traffic_and_op_counts_keyed_to_their_kernels_and_sources(monkeypatch):
    """The ncu-derived DRAM traffic and float32-op counts apply only to the kernel they were
    captured from, and only while its sources hash to the captured value."""
    cells = 1 << 20
    for mode, name in (("f32", "k_step_tma<float,dev,MC>"), ("dd", bench.KERNEL_NAMES[8]),
                       ("f64", "k_step_stream<double,plain,MC>")):
        t = bench.TRAFFIC_PER_CELL[mode]
        assert bench.kernel_sources_sha(t["sources"]) == t["sha"], mode   # captured from these sources
        assert bench.traffic_per_launch(mode, cells, name) == pytest.approx(t["bytes"] * cells)
    # other kernels of the same precision get no traffic figure
    assert bench.traffic_per_launch("dd", cells, bench.KERNEL_NAMES[9]) is None
    assert bench.traffic_per_launch("f32", cells, "k_step<float,dev,MC,256>") is None
    assert bench.dd_fp32_ops_per_cell() == bench.DD_FP32_OPS["ops"]
    # a source change voids both
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda names: "0" * 16)
    assert bench.traffic_per_launch("dd", cells, bench.KERNEL_NAMES[8]) is None
    assert bench.dd_fp32_ops_per_cell() is None
