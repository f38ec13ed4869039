"""bench.py's multi-rank path on CPU: two gloo ranks launched as torchrun
would (RANK / WORLD_SIZE / MASTER_* in the environment). The job's time is
the slowest rank's (max over ranks), its work the sum over ranks, and a
rank other than 0 leaves the reference arm without doing any work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, lr = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    mx = bench.max_over_ranks(10.0 * (r + 1), dist, "cpu")
    sm = bench.sum_over_ranks(3.0, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    ref = bench.main(["--impl", "reference"]) if r != 0 else None
    out.put((r, w, mx, sm, ref))


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, mx, sm, ref in res:
        assert w == world
        assert mx == 20.0          # slowest rank's value
        assert sm == 6.0           # work of both ranks
    assert res[1][4] == 0          # rank 1 leaves the reference arm at once
