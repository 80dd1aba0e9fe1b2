"""The multi-GPU path is replicas (independent instances per rank, weak
scaling, no data-path collective).  Its host logic -- the max-over-ranks
timing reduction, the whole-job value, and the reference arm's non-zero ranks
leaving without work -- runs here as world-size-2 gloo ranks on CPU."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    local = [10.0 + 5.0 * rank, 2.0 - rank]  # rank 1 is slower in the first value only
    got = bench.reduce_max(local, world)
    value = bench.weak_scaling_value(world, 1 << 20, 3, got[0])
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, value))


def test_max_over_ranks_and_whole_job_value():
    world, port = 2, _free_port()
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in out:
        assert got == [15.0, 2.0]                       # both ranks see the maxima
        assert value == pytest.approx(2 * (1 << 20) * 3 / 0.015)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max([3.0, 4.0], 1) == [3.0, 4.0]


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "1"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_traffic_figures_only_for_unchanged_kernel_sources(monkeypatch):
    """The DRAM traffic the bench line reports comes from an ncu capture; it is
    reported only while every source file of the kernel still has the digest
    recorded with the capture, and a changed source makes it null."""
    import bench
    for name, ent in bench.MEASURED_TRAFFIC.items():
        assert ent["sources"][0].endswith(".cu")
        want = ent["bytes"] if bench.source_digest(ent["sources"]) == ent["sha256"] else None
        assert bench.measured_traffic(name) == want
        stale = dict(ent, sha256="0" * 16)
        monkeypatch.setitem(bench.MEASURED_TRAFFIC, name, stale)
        assert bench.measured_traffic(name) is None
    assert bench.measured_traffic("no_such_kernel") is None
