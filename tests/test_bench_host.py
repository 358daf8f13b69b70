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


def test_run_serving_end_to_end_with_a_fake_server():
    """bench.run_serving's submission loop and statistics against a stand-in for the server
    binding (the real one needs a GPU): results come back in ticket order, one per request."""
    import types
    import bench

    class FakeServer:
        def __init__(self, budget, max_slots, steps_per_launch, queue_capacity):
            self.reqs = []

        def submit(self, req):
            self.reqs.append(req)
            return len(self.reqs) - 1

        def wait(self, ticket, timeout):
            r = self.reqs[ticket]
            return types.SimpleNamespace(latency_ms=10.0 + ticket, queue_ms=1.0,
                                         cells=r["cells"], nsteps=r["nsteps"], status=0)

        def close(self):
            pass

    def make_request(nx, nk, lo, hi, lk, dt, nsteps, nuclei, packets, precision):
        return {"cells": nx ** 3 * nk ** 3, "nsteps": nsteps, "precision": precision}

    ch = types.SimpleNamespace(Server=FakeServer, make_request=make_request)
    out = bench.run_serving(ch, n_req=6, rate=1e6, seed=7, nx_choices=(16,), nk_choices=(16,),
                            steps=(10, 12), precisions=(0, 1), budget=1 << 30, max_slots=2, spl=5)
    assert out["requests"] == 6 and out["failed"] == 0 and out["rate_per_s"] == 1e6
    assert out["p99_ms"] == 15.0 and out["cell_updates_per_s"] > 0
    specs = bench.serving_specs(7, 6, (16,), (16,), (10, 12), (0, 1))
    if len({s["precision"] for s in specs}) > 1:
        assert sum(b["requests"] for b in out["by_precision"].values()) == 6


def test_deviation_metrics_match_the_oracle_error_metrics():
    """The bench reduces eps_inf and eps_2 (Sec. 5) on the device; on CPU tensors its helper
    gives the pinned oracle's values."""
    import numpy as np
    import bench
    from oracle import chasm_oracle as O
    prob = O.Problem(nx=(5, 4, 6), nk=4, x_lo=(-2.0, -1.0, -3.0), x_hi=(2.0, 1.4, 2.0), lk=1.4)
    rng = np.random.default_rng(11)
    a = rng.standard_normal(prob.shape)
    b = a + 1e-3 * rng.standard_normal(prob.shape)
    got = bench.deviation_metrics(torch, torch.from_numpy(a).float(), torch.from_numpy(b),
                                  O.cell_volume(prob))
    ref = O.errors(b, a.astype(np.float32).astype(np.float64), prob)
    assert got == pytest.approx(ref, rel=1e-12)


def test_serving_both_forms_serve_the_same_stream():
    """serving_both submits the same requests (grid, steps, potential, packet) in each form."""
    import types
    import bench

    seen = {0: [], 1: []}

    class FakeServer:
        def __init__(self, budget, max_slots, steps_per_launch, queue_capacity):
            self.reqs = []

        def submit(self, req):
            self.reqs.append(req)
            seen[req["precision"]].append({k: v for k, v in req.items() if k != "precision"})
            return len(self.reqs) - 1

        def wait(self, ticket, timeout):
            r = self.reqs[ticket]
            return types.SimpleNamespace(latency_ms=10.0 + ticket + 100 * r["precision"],
                                         queue_ms=0.0, cells=r["cells"], nsteps=r["nsteps"],
                                         status=0)

        def close(self):
            pass

    def make_request(nx, nk, lo, hi, lk, dt, nsteps, nuclei, packets, precision):
        return {"cells": nx ** 3 * nk ** 3, "nsteps": nsteps, "precision": precision,
                "nuclei": nuclei, "packets": packets}

    ch = types.SimpleNamespace(Server=FakeServer, make_request=make_request, FP32_MIXED=0, FP64=1)
    out = bench.serving_both(ch, n_req=5, rate=1e6, steps=(10, 15))
    assert seen[0] == seen[1] and len(seen[0]) == 5
    assert out["fp32_mixed"]["requests"] == out["fp64"]["requests"] == 5
    assert out["p99_ms_fp32_mixed_vs_fp64"] == [14.0, 114.0]
