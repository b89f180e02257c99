"""Multi-rank host logic of bench.py (replicas): max/sum over ranks, on CPU with gloo."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    assert bench.env_rank() == (rank, rank, world)
    mx = bench.max_over_ranks(1.5 + rank, world)
    sm = bench.sum_over_ranks(10.0 * (rank + 1), world)
    out.put((rank, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
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
    for rank, mx, sm in res:
        assert mx == 2.5  # the slowest rank's time
        assert sm == 30.0  # work of all ranks


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.sum_over_ranks(3.0, 1) == 3.0


def test_reference_arm_runs_on_a_small_workload(capsys, monkeypatch):
    # the CPU reference arm (the oracle) on the small full-space workload
    sys.path.insert(0, ROOT)
    import json

    import bench

    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "cfg1", "--steps", "1",
                                      "--warmup", "3", "--ref-step-seconds", "0.3"])
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench.main() == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
