"""Host logic of bench.py's multi-rank path (replicas only): the whole-job value takes the
slowest rank's time, over a world-size-2 gloo group on the CPU; the reference arm prints only
on rank 0."""
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
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, tot = bench.replica_throughput(10.0 + 5.0 * rank, 4, 1e9, dist, "cpu")
        q.put((rank, value, tot))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_takes_the_slowest_rank():
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
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, value, tot in res:
        assert tot == pytest.approx(15.0)  # max over ranks (10 ms and 15 ms)
        assert value == pytest.approx(2 * 4 * 1e9 / 0.015 / 1e9)  # both ranks' work / that time


def test_replica_throughput_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, tot = bench.replica_throughput(20.0, 5, 2e9)
    assert tot == 20.0 and value == pytest.approx(5 * 2e9 / 0.02 / 1e9)


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup, gpus = 1, 0, 2
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""


def test_profile_traffic_needs_the_profiled_depth():
    """The roofline's `traffic` comes from a committed ncu summary only at the fused depth
    that summary captured (and only while the kernel sources match its sha)."""
    import re
    import bench
    prof_dir = os.path.join(ROOT, "profiles")
    checked = 0
    for name in sorted(os.listdir(prof_dir)):
        with open(os.path.join(prof_dir, name)) as f:
            text = f.read()
        m_t = re.search(r"fusion_depth:\s*([0-9]+)", text)
        m_b = re.search(r"dram_bytes_per_launch_scaled:\s*([0-9.eE+]+)", text)
        if not (m_t and m_b):
            continue
        depth, recorded = int(m_t.group(1)), float(m_b.group(1))
        got = bench._profile_traffic(depth, name)
        assert got is None or got == recorded
        assert bench._profile_traffic(depth + 1, name) is None
        checked += 1
    assert checked >= 1
