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


def test_oracle_sample_times_only_the_steps_after_warmup():
    import bench

    t = bench.cpu_oracle_sample(6, 4, 2, 3, timeout=300, warmup=1)
    assert 0.0 < t < 30.0


def test_oracle_on_several_cores_runs_released_replicas():
    """Two single-threaded oracle processes (independent replicas), released together: the
    slowest one's time and the node updates of both."""
    import bench

    t, nodes = bench.cpu_oracle_run(6, 4, 2, procs=2, warmup=1, timeout=300)
    assert 0.0 < t < 30.0 and nodes == 2 * 6 ** 3 * 2
    assert 1 <= bench.oracle_procs(128) <= (os.cpu_count() or 1)
    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()


def test_reference_line_keeps_the_contract(monkeypatch, capsys):
    """The reference arm (the FP64 oracle on the host cores) prints one JSON line with the main
    arm's metric, unit and config, impl = reference, its CPU baseline (cores used, CPU model)
    and an end-to-end object with no host-device traffic; a box too slow for the time budget
    is replaced by the largest sub-box that fits, and the line says so."""
    import argparse
    import json

    import bench

    calls = []

    def fake(L, N, steps, procs=1, warmup=0, seed=bench.SEED, timeout=900.0):
        calls.append((L, N, steps, procs, warmup))
        return 1e-6 * L ** 3 * steps, procs * L ** 3 * steps  # 2.1 s per step at L = 128, 0.26 s at L = 64
    monkeypatch.setattr(bench, "cpu_oracle_run", fake)
    monkeypatch.setattr(bench, "oracle_procs", lambda L: 4)
    bench.run_reference(argparse.Namespace(steps=20, warmup=5))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "MLUPS"
    assert line["steps"] == 20 and line["warmup"] == 5 and line["higher_is_better"] is True
    assert line["config"]["workload"] == bench.workload_name()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 4 and cb["cpu_model"]
    # budget 150 s / 25 steps = 6 s per step: L = 128 (2.1 s) fits
    assert calls[-1] == (bench.L_BENCH, bench.N_BENCH, 20, 4, 5)
    assert line["value"] == pytest.approx(4.0)  # 4 L^3 / (1e-6 L^3) / 1e6
    calls.clear()
    bench.run_reference(argparse.Namespace(steps=200, warmup=50))  # 0.6 s per step: L = 64
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert calls[-1] == (64, bench.N_BENCH, 200, 4, 50)
    assert "L=64 sub-box" in line["cpu_baseline"]["sample"]
