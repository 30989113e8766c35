"""Multi-process (world size 2, gloo, CPU) tests of the benchmark's N > 1 logic.

The path shards by instance: every rank runs an independent replica and the
only collectives are the timing ones (barrier, max of the timed milliseconds,
sum of the units processed).  The reference arm runs on rank 0 alone.
"""
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


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_env()
    assert (w, r, local) == (ws, rank, rank)
    bench.dist_init(ws, "gloo")
    bench.barrier(ws)
    # rank r timed 10 + r ms and processed 100 * (r + 1) units
    ms, units = bench.aggregate(10.0 + rank, 100.0 * (rank + 1), ws)
    # the reference arm: ranks other than 0 return at once without output
    rc = bench.run_reference(bench.parse(["--impl", "reference"])) if rank != 0 else 0
    out.put((rank, ms, units, rc))
    dist.destroy_process_group()


def test_world_size_2_timing_collectives_and_reference_rank_gate():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, rc in res:
        assert ms == 11.0          # max over ranks
        assert units == 300.0      # sum over ranks
        assert rc == 0


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.5, 7.0, 1) == (3.5, 7.0)
