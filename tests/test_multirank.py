"""Multi-rank host logic of bench.py on CPU with the gloo backend (world size 2): instances are
sharded across ranks with disjoint seeds, and the whole-job throughput is the sum of all ranks'
solves over the slowest rank's time (no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    seeds = bench.test_seeds(rank, 4)
    # rank r solves 10 + r instances in 2 + r seconds
    v = bench.job_throughput(ws, 10.0 + rank, 2.0 + rank)
    mx = bench.max_over_ranks(ws, float(rank))
    sm = bench.sum_over_ranks(ws, 1.0)
    out.put((rank, seeds, v, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_aggregation():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds0, seeds1 = res[0][1], res[1][1]
    assert not set(seeds0) & set(seeds1) and len(seeds0) == 4
    for rank, _, v, mx, sm in res:
        assert v == pytest.approx((10.0 + 11.0) / 3.0)   # all solves / slowest rank's time
        assert mx == 1.0 and sm == 2.0
