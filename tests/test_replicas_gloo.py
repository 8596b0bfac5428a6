"""Whole-job aggregation of bench.py's replicas, run as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r searched the same 3 roots (m edges each) in 1, 2, 4 ms times (r+1)
    m = [1_000_000, 2_000_000, 4_000_000]
    t = [(r + 1) * x for r, x in [(rank, 1.0), (rank, 2.0), (rank, 4.0)]]
    v = bench.replica_hm_gteps(dist, world, m, t)
    mx = bench._max_over_ranks(dist, float(rank * 10 + 1))
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, v, mx))


def test_replica_value_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank (rank 1): sum t/m = 3 x (2 ms / 1e6) = 6e-9 s per edge;
    # 2 ranks x 3 searches / 6e-9 s = 1e9 TEPS = 1 GTEPS
    for _, v, mx in res:
        assert abs(v - 1.0) < 1e-9
        assert mx == 11.0
