"""Host-side logic of bench.py on the CPU: the multi-rank aggregation (two gloo ranks) and the
seeded serving stream."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate_ranks(10.0 * (rank + 1), cells=1000, steps=3, dist=dist)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 20.0                                  # the slowest rank
        assert value == pytest.approx(2 * 1000 * 3 / 0.020)


def test_single_process_aggregation_is_the_local_rate():
    import bench
    ms, value = bench.aggregate_ranks(8.0, cells=500, steps=4)
    assert ms == 8.0 and value == pytest.approx(500 * 4 / 0.008)


def test_serving_stream_is_seeded_and_keeps_nuclei_off_the_nodes():
    import bench
    a = bench.serving_specs(2205, 64, (16, 24, 32), (16, 32), (10, 100), (0, 1))
    b = bench.serving_specs(2205, 64, (16, 24, 32), (16, 32), (10, 100), (0, 1))
    assert a == b
    assert {s["nx"] for s in a} == {16, 24, 32} and {s["nk"] for s in a} == {16, 32}
    assert all(10 <= s["nsteps"] <= 100 for s in a)
    for s in a:
        h = 2 * s["L"] / (s["nx"] - 1)
        for pos, _ in s["nuclei"]:
            assert all(-2 <= c <= 2 for c in pos)
            for c in pos:
                t = (c + s["L"]) / h
                assert abs(t - round(t)) * h >= h / 4 - 1e-12


def test_serving_stats_percentiles_and_per_precision_split():
    import bench
    rows = [(0, float(10 * i), 1.0, 100, 0) for i in range(1, 11)] + \
           [(1, float(1000 + i), 2.0, 50, 0) for i in range(1, 5)]
    st = bench.serving_stats(rows, wall=2.0)
    assert st["requests"] == 14 and st["failed"] == 0
    assert st["p50_ms"] == 70.0                 # nearest rank 7 of 14
    assert st["p99_ms"] == 1004.0
    assert st["cell_updates_per_s"] == pytest.approx((10 * 100 + 4 * 50) / 2.0)
    fp32, fp64 = st["by_precision"]["fp32_mixed"], st["by_precision"]["fp64"]
    assert (fp32["requests"], fp32["p50_ms"], fp32["p99_ms"]) == (10, 50.0, 100.0)
    assert (fp64["requests"], fp64["p50_ms"], fp64["p99_ms"]) == (4, 1002.0, 1004.0)
    one = bench.serving_stats(rows[:10], wall=1.0)
    assert "by_precision" not in one and one["p99_ms"] == 100.0
