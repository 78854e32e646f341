"""The N > 1 path of bench.py, on CPU: two ranks over gloo (127.0.0.1).
Replicas only — no data-path collective — so what the ranks share is the
timing: the job's time is the slowest rank's (max over ranks), the value is
the units of all ranks over that time, and the reference arm runs on rank 0
alone while the other ranks exit without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = bench.dist_setup()
        elapsed = 1.0 + 0.5 * rank           # rank 1 is the slow one
        job = bench.max_over_ranks(elapsed, w, torch.device("cpu"))
        value = bench.job_rate(1000.0, 10, w, job)

        class Args:
            steps, warmup = 1, 0
        ref = bench.run_reference(Args(), bench.workload("small")) if rank != 0 else None
        dist.barrier()
        out.put((rank, w, r, local, job, value, ref))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got.sort()
    for rank, w, r, local, job, value, ref in got:
        assert (w, r, local) == (2, rank, rank)
        assert job == 1.5                      # the slowest rank's time on every rank
        assert value == 1000.0 * 10 * 2 / 1.5  # units of both ranks over that time
    assert got[1][6] == 0                      # rank 1 leaves the reference arm without work


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.job_rate(100.0, 3, 1, 2.0) == 150.0
