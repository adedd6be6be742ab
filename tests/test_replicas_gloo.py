"""The multi-GPU path is replicas only (one independent problem per rank, no data-path collective): the
benchmark's host logic across ranks, run as two gloo ranks on the CPU.  Every rank must see the same
slowest-rank time and the same whole-job rate (units of all ranks over the slowest rank's time), and
the reference arm must leave ranks other than 0 without work."""
import os
import socket
import sys

import multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    try:
        import bench
        d = bench.Dist()
        d.init("gloo")
        d.barrier()
        slowest = d.max(0.25 * (rank + 1))
        rate, sec = bench.whole_job_rate(d, 1000.0, 0.5 * (rank + 1))
        ref = bench.run_reference(None, d, None, None) if rank != 0 else "rank 0 not run"
        d.barrier()
        d.done()
        q.put((rank, slowest, rate, sec, ref))
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e)))


def test_two_gloo_ranks_agree_on_slowest_time_and_whole_job_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rec in out:
        assert len(rec) == 5, rec
        rank, slowest, rate, sec, ref = rec
        assert slowest == 0.5                      # max over ranks of 0.25 (rank 0) and 0.5 (rank 1)
        assert sec == 1.0 and rate == 2 * 1000.0 / 1.0
        if rank != 0:
            assert ref is None                     # the oracle arm runs on rank 0 only
