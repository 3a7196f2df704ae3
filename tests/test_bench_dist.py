"""The multi-process side of bench.py on CPU: world size 2 over gloo (the GPU
runs use one process per GPU over NCCL with the same code). Every rank runs
its own replica; the whole-job rate is the units of all ranks over the
slowest rank's time, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.barrier()
    # rank r processed 100 (r + 1) units in 10 (r + 1) ms
    rate, ms_max = bench.whole_job_rate(d, 100.0 * (rank + 1), 10.0 * (rank + 1))
    zero_rate, zero_ms = bench.whole_job_rate(d, 0.0, 0.0)
    q.put((rank, d.world, rate, ms_max, d.reduce(float(rank), "MAX"), zero_rate, zero_ms))
    d.barrier()
    d.close()


def test_two_rank_replicas_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, w, rate, ms_max, rmax, zero_rate, zero_ms in out:
        assert w == 2
        assert ms_max == 20.0                       # the slowest rank's time
        assert rate == pytest.approx(300.0 / 0.020)  # all ranks' units / max time
        assert rmax == 1.0
        assert zero_rate == 0.0 and zero_ms == 0.0


def test_single_process_dist_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    d = bench.Dist()
    assert d.world == 1 and d.rank == 0
    rate, ms = bench.whole_job_rate(d, 50.0, 5.0)
    assert rate == pytest.approx(10000.0) and ms == 5.0
