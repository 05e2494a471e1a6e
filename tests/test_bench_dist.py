"""Host logic of bench.py's multi-rank mode on the CPU (gloo, world size 2).

With N ranks the bench runs N independent replicas of the workload: no data
crosses ranks, the timed region is bracketed by barriers, the step time is the
maximum over ranks and only rank 0 prints.  This checks those pieces without a
GPU, and the summary of the nvidia-smi clock samples the bench takes during the
timed region (median SM clock, throttle reasons seen active).
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        ms = bench.allreduce_max(world, 10.0 + 5.0 * rank)     # rank 1 is the slow one
        bench.barrier(world)
        q.put((rank, ms))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_gloo():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=5) for _ in range(2))
    assert got == {0: 15.0, 1: 15.0}


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    bench.barrier(1)
    assert bench.allreduce_max(1, 3.25) == 3.25


def test_clock_summary_from_nvidia_smi_lines():
    sys.path.insert(0, ROOT)
    import bench
    text = "\n".join([
        "0, 2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1398.1, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 905.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",     # unreadable sample: skipped
        "garbage line",
    ])
    c = bench.summarize_clocks(text)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    hot = "0, 1500, 2070, 1400, 0x48, Active, Not Active, Active, Not Active"
    assert bench.summarize_clocks(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarize_clocks("") is None
