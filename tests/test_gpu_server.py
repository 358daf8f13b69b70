"""Continuous-batching server on the GPU: results are the same alone and in the mix, admission
respects the HBM budget, cancellation and queue limits work."""
import ctypes as C
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ch():
    import paper_2205_02380_gb300 as pkg
    pkg.chasm.lib()
    assert torch.cuda.is_available()
    return pkg


def request_specs():
    """Seeded mix of grids, precisions, nuclei and step counts (a small version of the serving
    stream: grids from {8,10,12}^3 x {8,16}^3, 1-2 protons in [-2,2]^3, one packet each)."""
    g = synth.SplitMix64(2205)
    specs = []
    for i in range(7):
        nx = [8, 10, 12][g.randint(0, 2)]
        nk = [8, 16][g.randint(0, 1)]
        nn = g.randint(1, 2)
        nuc = [((g.uniform(-2, 2), g.uniform(-2, 2), g.uniform(-2, 2)), 1.0) for _ in range(nn)]
        pk = [synth.packet([g.uniform(-2, 2) for _ in range(3)],
                           [g.uniform(-1, 1) for _ in range(3)])]
        specs.append(dict(nx=nx, nk=nk, nuclei=nuc, packets=pk, nsteps=g.randint(3, 9),
                          precision=i % 2, L=6.0, lk=4.0, dt=0.025))
    return specs


def run_alone(ch, sp):
    with ch.Solver(sp["nx"], sp["nk"], -sp["L"], sp["L"], sp["lk"], nuclei=sp["nuclei"],
                   precision=sp["precision"]) as s:
        dt = torch.float64 if sp["precision"] == ch.FP64 else torch.float32
        f = torch.empty((sp["nx"],) * 3 + (sp["nk"],) * 3, device="cuda", dtype=dt)
        s.init_gaussians(f, sp["packets"])
        s.step(f, sp["dt"], sp["nsteps"])
        m, e = s.moments(f)
        return f.cpu().numpy(), m, e


def make_req(ch, sp, out):
    return ch.make_request(sp["nx"], sp["nk"], -sp["L"], sp["L"], sp["lk"], sp["dt"], sp["nsteps"],
                           nuclei=sp["nuclei"], packets=sp["packets"], precision=sp["precision"],
                           fout_ptr=out.ctypes.data)


def test_results_are_identical_alone_and_in_the_mix(ch):
    specs = request_specs()
    outs = [np.zeros((sp["nx"],) * 3 + (sp["nk"],) * 3,
                     dtype=np.float64 if sp["precision"] == ch.FP64 else np.float32) for sp in specs]
    srv = ch.Server(4 << 30, max_slots=4, steps_per_launch=2)
    try:
        reqs = [make_req(ch, sp, o) for sp, o in zip(specs, outs)]
        tickets = [srv.submit(r) for r in reqs]
        res = [srv.wait(t, 300.0) for t in tickets]
    finally:
        srv.close()
    for sp, o, r in zip(specs, outs, res):
        assert r.status == 0
        assert r.nsteps == sp["nsteps"]
        assert r.latency_ms >= r.run_ms >= 0.0
        f, m, e = run_alone(ch, sp)
        assert np.array_equal(o, f), "result differs between the mix and a lone run"
        assert r.mass == m and r.energy == e


def test_admission_respects_the_budget_and_slots(ch):
    import time
    sp = dict(nx=12, nk=16, nuclei=[((0.0, 0.0, 0.0), 1.0)], packets=[synth.packet((0, 0, 0), (0, 0, 0))],
              nsteps=30, precision=ch.FP32_MIXED, L=6.0, lk=4.0, dt=0.025)
    per = ch.chasm.workspace_bytes(12, 16, nuclei=sp["nuclei"]) + 12 ** 3 * 16 ** 3 * 4
    srv = ch.Server(int(2.5 * per), max_slots=8, steps_per_launch=1)
    try:
        outs = [np.zeros((12,) * 3 + (16,) * 3, dtype=np.float32) for _ in range(5)]
        tickets = [srv.submit(make_req(ch, sp, o)) for o in outs]
        peak_running, peak_bytes = 0, 0
        t0 = time.time()
        while time.time() - t0 < 120:
            q, r, b = srv.stats()
            peak_running, peak_bytes = max(peak_running, r), max(peak_bytes, b)
            if q == 0 and r == 0:
                break
            time.sleep(0.002)
        res = [srv.wait(t, 60.0) for t in tickets]
    finally:
        srv.close()
    assert all(r.status == 0 for r in res)
    assert 1 <= peak_running <= 2          # only two requests fit in 2.5x one request's bytes
    assert peak_bytes <= int(2.5 * per)
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])  # same request, same answer, whatever the interleaving


def test_cancel_and_queue_limits(ch):
    sp = dict(nx=10, nk=16, nuclei=[((0.1, 0.0, 0.0), 1.0)], packets=[synth.packet((0, 0, 0), (0, 0, 0))],
              nsteps=400, precision=ch.FP64, L=6.0, lk=4.0, dt=0.02)
    srv = ch.Server(8 << 30, max_slots=1, steps_per_launch=1, queue_capacity=2)
    try:
        o = np.zeros((10,) * 3 + (16,) * 3)
        import time
        t1 = srv.submit(make_req(ch, sp, o))
        t0 = time.time()
        while srv.stats()[1] < 1 and time.time() - t0 < 30:   # wait until t1 holds the slot
            time.sleep(0.001)
        t2 = srv.submit(make_req(ch, sp, o))
        t3 = srv.submit(make_req(ch, sp, o))
        with pytest.raises(ch.ChasmError) as e:
            srv.submit(make_req(ch, sp, o))          # t2, t3 fill the queue of capacity 2
        assert e.value.code == ch.chasm.EAGAIN
        srv.cancel(t3)
        srv.cancel(t1)
        r1 = srv.wait(t1, 60.0)
        r3 = srv.wait(t3, 60.0)
        assert r3.status == ch.chasm.ECANCELED
        assert r1.status == ch.chasm.ECANCELED
        srv.cancel(t2)
        assert srv.wait(t2, 60.0).status == ch.chasm.ECANCELED
    finally:
        srv.close()
