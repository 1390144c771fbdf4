"""The benchmark's multi-rank path on CPU: world_size 2 over gloo.  Every rank runs an
independent replica (no data-path collective); the job throughput is the units of all ranks
over the MAX of the ranks' timed regions."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    ws_, rank_, local_ = bench.dist_env()
    seconds = [2.0, 3.0][rank]  # rank 1 is the slow one
    value, tmax = bench.aggregate_throughput(100.0, seconds, ws_)
    q.put((rank_, local_, value, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_uses_max_time_and_sums_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, local, value, tmax in res:
        assert tmax == pytest.approx(3.0)
        assert value == pytest.approx(2 * 100.0 / 3.0)
    assert [r[0] for r in res] == [0, 1]


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(1.5, 1) == 1.5
    v, t = bench.aggregate_throughput(10.0, 2.0, 1)
    assert (v, t) == (5.0, 2.0)
