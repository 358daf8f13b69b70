"""Benchmark: 6-D cell-updates per second of one Strang step of the CHASM scheme on GB300.

Headline workload (`value`): the two-centre Coulomb problem V = -1/|x - a| - 1/|x + a|,
a = (0.7, 0, 0), on 64^3 x 32^3 cells over [-16,16]^3 x [-4,4)^3 (8.6e9 cells, 34 GB per FP32
copy of f), initial f the seeded mixture of two unit-mass packets (SplitMix64 seed 2205),
dt = 0.02, FP32-mixed form: the largest of the paper-shaped workloads that fits one GPU.  The FP64
form is timed on the largest workload whose FP64 table form fits one GPU, the electron-proton case
48^3 x 32^3 on [-12,12]^3 ("fp64", next to the FP32-mixed form on the same workload), and the
hydrogen 1s stationarity test 32^3 x 32^3 runs its 40 steps in both forms ("stationarity").

Prints ONE JSON line (rank 0).  Under torchrun with N > 1 every rank runs its own replica of the
workload on its own GPU (no data-path collective) and `value` is the sum over ranks of cells
updated divided by the slowest rank's time ("scaling": "weak").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl chasm|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "6-D cell-updates/s per Strang step, FP32-mixed vs FP64 at stated L2 error"
UNIT = "cell-updates/s"

# The paper-shaped workloads (Sec. 5.2-5.4), all with hbar = m = 1 and L_k = 4.
#   init: ("gauss", seed or packet list) or ("1s", N_y)
WORKLOADS = {
    "two-centre": {
        "name": "two-centre 64^3x32^3 [-16,16]^3 x [-4,4)^3, V=-1/|x-a|-1/|x+a|, a=(0.7,0,0), "
                "seeded two-packet mixture (seed 2205), dt=0.02",
        "nx": 64, "nk": 32, "L": 16.0, "lk": 4.0, "dt": 0.02,
        "nuclei": [((0.7, 0.0, 0.0), 1.0), ((-0.7, 0.0, 0.0), 1.0)],
        "init": ("mixture", 2205)},
    "electron-proton": {
        "name": "electron-proton 48^3x32^3 [-12,12]^3 x [-4,4)^3, V=-1/|x|, packet at (-4,0,0) "
                "with k0=(1,0,0), dt=0.02",
        "nx": 48, "nk": 32, "L": 12.0, "lk": 4.0, "dt": 0.02,
        "nuclei": [((0.0, 0.0, 0.0), 1.0)],
        "init": ("packet", ((-4.0, 0.0, 0.0), (1.0, 0.0, 0.0)))},
    "hydrogen-1s": {
        "name": "hydrogen-1s 32^3x32^3 [-12,12]^3 x [-4,4)^3, V=-1/|x|, dt=0.025",
        "nx": 32, "nk": 32, "L": 12.0, "lk": 4.0, "dt": 0.025,
        "nuclei": [((0.0, 0.0, 0.0), 1.0)],
        "init": ("1s", 128)},
}
HEADLINE = "two-centre"
FP64_WORKLOAD = "electron-proton"
STATIONARITY = "hydrogen-1s"


def cells_of(W) -> int:
    return W["nx"] ** 3 * W["nk"] ** 3


def packets_of(W):
    """Initial packets of a Gaussian workload (synth's unit-mass packets)."""
    import synth
    kind, arg = W["init"]
    if kind == "mixture":
        return synth.two_packet_mixture(arg)
    if kind == "packet":
        return [synth.packet(*arg)]
    raise ValueError(kind)


# ------------------------------------------------------------------------------------------------
# algorithmic work of the dominant kernel (the P(dt) kernel of the table form: one launch = the
# four Horner stages of P(dt) over all x points; each stage applies Theta^T once)
def theta_flops_per_cell(nk: int) -> float:
    """Flops per cell of one application of Theta^T in the table form (all nuclei at once),
    complex FFTs of length n counted at 5 n log2 n:
      k3 forward   N^2 FFTs of length N on the twisted real line (twist 2 N^3)
      slab phase   6 N^2 zero-padded length-2N transforms (k2 and k1 forward, k1 and k2 inverse),
                   each two N-point FFTs plus the twist of the odd half (6 N), and the parity-
                   half sum of the 3 N^2 inverse ones (2 N each)
      symbol       (2N)^2 N products by i sigma (2 each)
      k3 inverse   N^2 FFTs of length N, conjugate twist and real part (3 N^3), Horner (2 N^3)
    all divided by N^3 (about 407 at N = 32)."""
    n = nk
    fft_n = 5 * n * math.log2(n)
    total = (2 * n * n * fft_n + 6 * n * n * (2 * fft_n + 6 * n) + 3 * n * n * 2 * n
             + 8 * n ** 3 + (2 + 3 + 2) * n ** 3)
    return total / n ** 3


def fp32_alu_peak_tflops(num_sms: int) -> float:
    """SMs (read from the device) x 128 FP32 lanes x 2 flops (FMA) x the maximum SM clock."""
    mhz = 2070.0
    try:
        mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        pass
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_hbm_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else the 6.8 TB/s
    fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def theta_source_hash() -> str:
    """Hash of the sources of the P(dt) kernel (the traffic figure is void once they change)."""
    h = hashlib.sha256()
    for name in ("k_theta_pk.cu", "fft_pk.cuh", "fft_reg.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2205_02380_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic():
    """DRAM bytes per launch of the Theta kernel from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "theta_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("source_sha256_16") != theta_source_hash():
        return None
    return d


# ------------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
def make_solver(ch, W, precision, stream, integrator=None):
    return ch.Solver(W["nx"], W["nk"], -W["L"], W["L"], W["lk"], nuclei=W["nuclei"],
                     precision=precision, stream=stream.cuda_stream, theta_form=ch.THETA_TABLE,
                     integrator=ch.STRANG if integrator is None else integrator)


def init_f(s, W, f):
    """Writes the workload's initial f on the GPU (chasm_init_gaussians / chasm_init_hydrogen_1s)."""
    kind, arg = W["init"]
    if kind == "1s":
        s.init_hydrogen_1s(f, n_y=arg)
    else:
        s.init_gaussians(f, packets_of(W))


def new_f(torch, W, dtp):
    return torch.empty((W["nx"],) * 3 + (W["nk"],) * 3, device="cuda", dtype=dtp)


def release(torch):
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def aggregate_ranks(ms_local: float, cells: int, steps: int, dist=None, device="cpu"):
    """Max over ranks of the timed milliseconds and the whole-job throughput: every rank updates
    `cells` cells per step (weak scaling), so value = world * cells * steps / max_ms."""
    world = 1
    ms = float(ms_local)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * cells * steps / (ms / 1e3)


def time_steps(torch, s, f, dt, steps, warmup, stream, dist):
    """W untimed steps, then exactly `steps` steps between CUDA events on the solver's stream,
    bracketed by barrier + synchronize.  Returns milliseconds and the kernels the library issued
    for the timed steps."""
    s.step(f, dt, warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n0 = s.launch_count()
    e0.record(stream)
    s.step(f, dt, steps)
    e1.record(stream)
    n1 = s.launch_count()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), n1 - n0


def time_pflow_launches(torch, s, f, dt, stream, reps):
    """Average duration of one launch of the P(dt) kernel (in the table form chasm_pflow is
    exactly one launch), on a copy of f, CUDA events on the solver's stream."""
    g = f.clone()
    s.pflow(g, dt)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        s.pflow(g, dt)
    e1.record(stream)
    torch.cuda.synchronize()
    del g
    return e0.elapsed_time(e1) / reps


def host_copy_gbs(torch, host, dev, stream):
    """Plain pinned host <-> device copy bandwidth of one f-sized buffer on this machine (GB/s,
    CUDA events), reported beside the end-to-end number: its copies move these bytes."""
    out = {}
    for name, dst, src in (("h2d", dev, host), ("d2h", host, dev)):
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            dst.copy_(src, non_blocking=True)
            e1.record(stream)
        torch.cuda.synchronize()
        out[name] = host.numel() * host.element_size() / (e0.elapsed_time(e1) / 1e3) / 1e9
    return out


def deviation_metrics(torch, a, b, vol):
    """eps_inf = max |a - b| and eps_2 = sqrt(sum (a - b)^2 vol) (the error metrics of Sec. 5,
    the integral as the grid sum times the cell volume), reduced in FP64 on a's device."""
    d = a.double() - b.double()
    return float(d.abs().max()), float(torch.sqrt((d * d).sum() * vol))


# ------------------------------------------------------------------------------------------------
# host-core baseline: the FP64 oracle on bounded pieces of the headline workload
def host_info() -> dict:
    """nproc and the CPU model of this machine."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            import platform
            model = platform.processor() or platform.machine()
        except Exception:
            model = "unknown"
    return {"nproc": os.cpu_count() or 1, "cpu_model": model}


_T_CACHE = {}


def _oracle_task(task):
    """One independent piece of the oracle's step (runs in a worker process): ("A", k indices)
    advects the full x-cube at those k points by dt/2; ("P", x index) applies P(dt) on the full
    k-cube of one x point of the workload's initial data.  Returns (cells, seconds)."""
    import numpy as np

    import synth
    from oracle import chasm_oracle as O
    kind, wname, idx = task
    W = WORKLOADS[wname]
    nx, nk, L, lk, dt = W["nx"], W["nk"], W["L"], W["lk"], W["dt"]
    prob = O.Problem(nx=(nx,) * 3, nk=nk, x_lo=(-L,) * 3, x_hi=(L,) * 3, lk=lk,
                     nuclei=W["nuclei"])
    if kind == "A":
        # the spline transform and the 64-tap sum cost the same for any data: smooth surrogate
        ks = prob.ks()
        g = np.exp(-0.05 * prob.xs(0) ** 2)
        cube = (g[:, None, None] * g[None, :, None] * g[None, None, :])[..., None, None, None]
        a, b, c = idx
        t0 = time.perf_counter()
        O.advect(cube, prob, 0.5 * dt, kaxes=(ks[a:a + 1], ks[b:b + 1], ks[c:c + 1]))
        return nx ** 3, time.perf_counter() - t0
    xs = prob.xs(0)
    x = np.array([xs[idx[0]], xs[idx[1]], xs[idx[2]]])
    # the initial data at the one x point (a 2-point grid starting there, first node kept)
    if W["init"][0] == "1s":
        f1 = synth.wigner_1s((2, 2, 2), nk, tuple(x), tuple(x + 1.0), lk, n_y=W["init"][1])
    else:
        f1 = synth.gaussian_packets((2, 2, 2), nk, tuple(x), tuple(x + 1.0), lk, packets_of(W))
    f1 = f1[:1, :1, :1]
    key = (nk, lk)
    if key not in _T_CACHE:   # T is computed once per handle on the GPU side as well
        _T_CACHE[key] = O.tkm_tensor(nk, lk)
    T = _T_CACHE[key]
    t0 = time.perf_counter()
    O.pflow_coulomb(f1.reshape(1, nk, nk, nk), prob, dt, T, xpts=x[None])
    return nk ** 3, time.perf_counter() - t0


def oracle_pool(workers: int):
    """A pool of `workers` spawned processes (no CUDA state is inherited) for oracle_sample."""
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def oracle_sample(wname: str, workers: int, n_a: int, n_p: int, seed: int = 2205, ex=None) -> dict:
    """Times the oracle on n_a k points of A(dt/2) (full x-cube each) and n_p x points of P(dt)
    (full k-cube each), spread over `workers` processes (spawned, one thread each); the pieces are
    independent, so the wall time of each batch gives that substep's cell rate on `workers` cores.
    Cell-update time = 2 t_A + t_P.  ex: an oracle_pool to reuse (else one is made)."""
    import numpy as np
    W = WORKLOADS[wname]
    nx, nk = W["nx"], W["nk"]
    rng = np.random.default_rng(seed)
    ka = [tuple(int(v) for v in rng.integers(0, nk, 3)) for _ in range(n_a)]
    # x points where f is not negligible: near the nuclei and the packet centres
    lo, h = -W["L"], 2 * W["L"] / (nx - 1)
    centres = [p for p, _ in W["nuclei"]]
    if W["init"][0] != "1s":
        centres += [pk["x0"] for pk in packets_of(W)]
    xp = []
    for i in range(n_p):
        c = centres[i % len(centres)]
        xp.append(tuple(int(min(nx - 1, max(0, round((c[d] - lo) / h) + rng.integers(-2, 3))))
                        for d in range(3)))
    tasks_a = [("A", wname, k) for k in ka]
    tasks_p = [("P", wname, x) for x in xp]
    if workers == 1:
        t0 = time.perf_counter()
        ra = [_oracle_task(t) for t in tasks_a]
        wa = time.perf_counter() - t0
        t0 = time.perf_counter()
        rp = [_oracle_task(t) for t in tasks_p]
        wp = time.perf_counter() - t0
    else:
        own = ex is None
        if own:
            ex = oracle_pool(workers)
        try:
            list(ex.map(_oracle_task, [("P", wname, xp[0])] * workers))   # imports, T, warm
            t0 = time.perf_counter()
            ra = list(ex.map(_oracle_task, tasks_a))
            wa = time.perf_counter() - t0
            t0 = time.perf_counter()
            rp = list(ex.map(_oracle_task, tasks_p))
            wp = time.perf_counter() - t0
        finally:
            if own:
                ex.shutdown()
    tA = wa / sum(c for c, _ in ra)
    tP = wp / sum(c for c, _ in rp)
    return {"value": 1.0 / (2 * tA + tP), "t_a_us": tA * 1e6, "t_p_us": tP * 1e6,
            "cpu_s": sum(t for _, t in ra) + sum(t for _, t in rp)}


def cpu_baseline_run(wname: str, repeats: int = 3) -> dict:
    """The oracle on all host cores and on one core, median of `repeats` bounded samples each."""
    info = host_info()
    n = info["nproc"]
    W = WORKLOADS[wname]
    out = {"unit": UNIT, "kind": "oracle", "cores": n, "cpu_model": info["cpu_model"],
           "nproc": n}
    with oracle_pool(n) as ex:
        runs_all = [oracle_sample(wname, n, n_a=2 * n, n_p=8 * n, seed=2205 + r, ex=ex)
                    for r in range(repeats)]
    runs_one = [oracle_sample(wname, 1, n_a=2, n_p=8, seed=2205 + r) for r in range(repeats)]
    med = lambda rs: statistics.median(r["value"] for r in rs)   # noqa: E731
    out["value"] = med(runs_all)
    out["value_all_cores"] = out["value"]
    out["value_1_core"] = med(runs_one)
    out["runs_all_cores"] = [r["value"] for r in runs_all]
    out["runs_1_core"] = [r["value"] for r in runs_one]
    out["sample"] = (
        f"FP64 numpy oracle on {W['name']}: per run A(dt/2) on the full {W['nx']}^3 x-cube at "
        f"2 k points per worker and P(dt) on the full {W['nk']}^3 k-cube at 8 x points per worker "
        f"(near the nuclei and packet centres), {n} spawned single-threaded workers (all cores) or "
        f"1; cell-update time 2 t_A + t_P; median of {repeats} runs each "
        f"(all cores: t_A {runs_all[0]['t_a_us']:.3f} us, t_P {runs_all[0]['t_p_us']:.3f} us per cell)")
    return out


def cpu_baseline(wname: str) -> dict:
    """Runs cpu_baseline_run in a fresh process with no GPU visible (threads pinned to one per
    worker) and returns its result."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                        "--workload", wname], capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": None, "kind": "oracle",
                "sample": "failed: " + r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


# ------------------------------------------------------------------------------------------------
def run_reference(args):
    """The oracle as it stands on all host cores: each step one bounded sample of the headline
    workload; value = median over the timed steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.update(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    info = host_info()
    n = info["nproc"]
    W = WORKLOADS[HEADLINE]
    per_step = []
    with oracle_pool(n) as ex:
        for i in range(args.warmup + args.steps):
            r = oracle_sample(HEADLINE, n, n_a=n, n_p=4 * n, seed=2205 + i, ex=ex)
            if i >= args.warmup:
                per_step.append(r["value"])
    value = statistics.median(per_step)
    sample = (f"FP64 numpy oracle on {W['name']}, {n} spawned single-threaded workers: per step "
              f"A(dt/2) on the full x-cube at {n} k points and P(dt) at {4 * n} x points; "
              f"cell-update time 2 t_A + t_P")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"], "cells": cells_of(W),
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                             "cpu_model": info["cpu_model"], "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_form(torch, ch, W, prec, steps, warmup, stream, dist, sampler=None, e2e_steps=0,
                 pflow_reps=1):
    """Times `steps` steps of one form on one workload (plus P(dt) launches and, with e2e_steps,
    the end-to-end host-buffer call).  Returns a dict."""
    cells = cells_of(W)
    dtp = torch.float32 if prec == ch.FP32_MIXED else torch.float64
    with torch.cuda.stream(stream):
        s = make_solver(ch, W, prec, stream)
        f = new_f(torch, W, dtp)
        init_f(s, W, f)
        m0, en0 = s.moments(f)
        if sampler:
            sampler.start()
        ms, launches = time_steps(torch, s, f, W["dt"], steps, warmup, stream, dist)
        clocks = sampler.stop() if sampler else None
        m1, en1 = s.moments(f)
        ms_t, value = aggregate_ranks(ms, cells, steps, dist, "cuda")
        entry = {"value": value, "ms_per_step": ms_t / steps, "steps": steps, "warmup": warmup,
                 "launches": launches, "mass_drift": (m1 - m0) / m0, "energy0": en0, "energy": en1}
        if clocks is not None:
            entry["clocks"] = clocks
        entry["pflow_ms"] = time_pflow_launches(torch, s, f, W["dt"], stream, pflow_reps)
        if e2e_steps:
            world = dist.get_world_size() if dist else 1
            # end-to-end through the C ABI with HOST buffers (pinned), copies included
            host = torch.empty(f.shape, dtype=dtp, pin_memory=True)
            host.copy_(f)
            hout = torch.empty_like(host, pin_memory=True)
            s.run_host(host.data_ptr(), hout.data_ptr(), W["dt"], 1)   # warm: buffer + graph
            runs = []
            for _ in range(3):   # median of three calls (host-side timing noise)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                s.run_host(host.data_ptr(), hout.data_ptr(), W["dt"], e2e_steps)
                runs.append(time.perf_counter() - t0)
            t_e2e = statistics.median(runs)
            entry["e2e"] = {"value": world * cells * e2e_steps / t_e2e, "unit": UNIT,
                            "h2d_bytes_per_step": s.f_bytes() / e2e_steps,
                            "d2h_bytes_per_step": (s.f_bytes() + 8) / e2e_steps,
                            "steps": e2e_steps, "wall_s": t_e2e,
                            "host_copy_gbs": host_copy_gbs(torch, host, f, stream)}
            del host, hout
        del f
        s.close()
    release(torch)
    return entry


def time_lpc1(torch, ch, W, stream, steps, warmup):
    """The paper's LPC1 integrator on a workload (FP32-mixed, table form): W untimed and `steps`
    timed steps, CUDA events on the solver's stream."""
    with torch.cuda.stream(stream):
        s = make_solver(ch, W, ch.FP32_MIXED, stream, ch.LPC1)
        f = new_f(torch, W, torch.float32)
        init_f(s, W, f)
        m0 = s.mass(f)
        ms, _ = time_steps(torch, s, f, W["dt"], steps, warmup, stream, None)
        m1 = s.mass(f)
        s.close()
        del f
    release(torch)
    return {"value": cells_of(W) * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "dtype": "f32", "workload": W["name"], "mass_drift": (m1 - m0) / m0,
            "note": "LPC1 (Sec. 2.2): 2 Theta applications and 6 advection passes per step (the "
                    "predictor and corrector base are formed inside the Theta kernel)"}


def stationarity_run(torch, ch, stream, steps):
    """Hydrogen 1s stationarity (Sec. 5.2): both forms from the same initial data for `steps`
    steps.  Reports the relative L2 distance of the FP32-mixed result from the FP64 result (the
    FP64 form is itself pinned to the FP64 oracle at 1e-12), and per form the drift of f from the
    stationary initial state (eps_inf, eps_2 of Sec. 5 and relative L2), of the mass and of the
    energy."""
    W = WORKLOADS[STATIONARITY]
    h = 2 * W["L"] / (W["nx"] - 1)
    vol = h ** 3 * (2 * W["lk"] / W["nk"]) ** 3
    out, finals = {}, {}
    with torch.cuda.stream(stream):
        for name, prec, dtp in (("fp64", ch.FP64, torch.float64), ("fp32", ch.FP32_MIXED, torch.float32)):
            s = make_solver(ch, W, prec, stream)
            f = new_f(torch, W, dtp)
            init_f(s, W, f)
            f0 = f.clone()
            m0, e0 = s.moments(f)
            s.step(f, W["dt"], steps)
            m1, e1 = s.moments(f)
            einf, e2 = deviation_metrics(torch, f, f0, vol)
            rel = float(torch.linalg.vector_norm((f - f0).double()) / torch.linalg.vector_norm(f0.double()))
            out[name] = {"eps_inf_vs_initial": einf, "eps_2_vs_initial": e2,
                         "rel_l2_vs_initial": rel, "mass_drift": (m1 - m0) / m0,
                         "energy0": e0, "energy_drift": (e1 - e0) / abs(e0)}
            del f0
            finals[name] = f
            s.close()
        a, b = finals["fp32"].double(), finals["fp64"]
        rel = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        del a, b, finals
    release(torch)
    out.update({"workload": W["name"], "steps": steps, "t_final": steps * W["dt"],
                "rel_l2_fp32_vs_fp64": rel, "tolerance": 1e-5,
                "mass_rel_diff_fp32_vs_fp64": None,
                "note": "the FP64 form is pinned to the FP64 oracle at <= 1e-12; eps_inf and eps_2 "
                        "against the initial state, which is stationary for the exact flow"})
    out["mass_rel_diff_fp32_vs_fp64"] = out["fp32"]["mass_drift"] - out["fp64"]["mass_drift"]
    return out


def run_chasm(args):
    import torch
    import paper_2205_02380_gb300 as ch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    ch.chasm.lib()
    num_sms = torch.cuda.get_device_properties(local).multi_processor_count
    W = WORKLOADS[HEADLINE]
    W64 = WORKLOADS[FP64_WORKLOAD]
    cells = cells_of(W)
    stream = torch.cuda.Stream()

    sampler = ClockSampler(local)
    r32 = measure_form(torch, ch, W, ch.FP32_MIXED, args.steps, args.warmup, stream, dist,
                       sampler=sampler, e2e_steps=max(1, args.e2e_steps), pflow_reps=3)
    clocks = r32.pop("clocks")
    r64 = measure_form(torch, ch, W64, ch.FP64, max(1, args.fp64_steps), 1, stream, dist)
    r64_32 = measure_form(torch, ch, W64, ch.FP32_MIXED, max(1, min(args.steps, 5)), 2, stream,
                          dist, pflow_reps=3)
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    stat = stationarity_run(torch, ch, stream, args.stat_steps) if args.stat_steps > 0 else None
    lpc1 = time_lpc1(torch, ch, W, stream, max(1, min(args.steps, 10)), 1) if not args.no_lpc1 else None
    serving = None
    if not args.no_serving:
        serving = serving_both(ch, n_req=args.bench_serve_requests, rate=args.bench_serve_rate,
                               steps=(10, 15))
    # the host-core baseline runs after the GPU measurements (its host allocations slowed the
    # pinned copies of the e2e call when made before them; the child process shares no CUDA state)
    base = cpu_baseline(HEADLINE) if (world == 1 and not args.no_cpu_baseline) else None

    nk = W["nk"]
    flops_launch = 4 * theta_flops_per_cell(nk) * cells
    achieved = flops_launch / (r32["pflow_ms"] / 1e3) / 1e12
    flops64 = 4 * theta_flops_per_cell(W64["nk"]) * cells_of(W64)
    achieved64 = flops64 / (r64["pflow_ms"] / 1e3) / 1e12
    peak = fp32_alu_peak_tflops(num_sms)
    try:
        fma32, fma64 = ch.chasm.fma_peaks()
        fma32x2 = ch.chasm.fma_peak_f32x2()
        fft_only = ch.chasm.fft_pk_rate() if nk == 32 else None
    except Exception:
        fma32 = fma64 = fma32x2 = fft_only = None
    tr = committed_traffic()
    e2e = r32.pop("e2e")
    line = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r32["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded two-packet mixture written on the GPU)",
        "config": {"workload": W["name"], "cells": cells, "global_batch": world,
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (f = %.1f GB)" % (cells * 4 / 1e9)},
        "headline_detail": r32,
        "fp64": {"workload": W64["name"], "cells": cells_of(W64), "dtype": "f64",
                 "value": r64["value"], "ms_per_step": r64["ms_per_step"], "steps": r64["steps"],
                 "pflow_ms": r64["pflow_ms"], "pflow_tflops": achieved64,
                 "pflow_frac_of_measured_fp64_fma": (achieved64 / fma64) if fma64 else None,
                 "fp32_mixed_same_workload": {"value": r64_32["value"],
                                              "ms_per_step": r64_32["ms_per_step"],
                                              "steps": r64_32["steps"]},
                 "fp32_over_fp64": r64_32["value"] / r64["value"]},
        "stationarity": stat,
        "lpc1": lpc1,
        "serving": serving,
        "roofline": {"kernel": "k_theta_pk<32> (P(dt): four Horner stages of Theta^T per x point, "
                               "table form, packed FP32)",
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_source": f"derived: {num_sms} SMs x 128 FP32 lanes x 2 x max SM clock",
                     "measured_fma_peak_tflops": fma32,
                     "frac_of_measured_fma_peak": (achieved / fma32) if fma32 else None,
                     "measured_packed_f32x2_fma_tflops": fma32x2,
                     "fft_only_tflops": fft_only,
                     "frac_of_fft_only": (achieved / fft_only) if fft_only else None,
                     "ms_per_launch": r32["pflow_ms"],
                     "flops_per_launch": flops_launch,
                     "traffic": (tr["dram_bytes_per_launch"] * cells / tr["cells"]) if tr else None},
        "e2e": e2e,
        "gpu_launches": r32["launches"],
        "clocks": clocks,
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serving_specs(seed, n_req, nx_choices, nk_choices, steps, precisions, L=12.0, lk=4.0):
    """Seeded request stream: grid from the choices, 1-2 protons uniform in [-2,2]^3 (redrawn when
    within h/4 of a node), an electron packet with centre in [-4,4]^3 and momentum in [-1.5,1.5]^3,
    steps uniform in the range, dt = 0.025."""
    import synth
    g = synth.SplitMix64(seed)
    specs = []
    for i in range(n_req):
        nx = nx_choices[g.randint(0, len(nx_choices) - 1)]
        nk = nk_choices[g.randint(0, len(nk_choices) - 1)]
        h = 2 * L / (nx - 1)
        nuc = []
        for _ in range(g.randint(1, 2)):
            while True:
                p = [g.uniform(-2, 2) for _ in range(3)]
                if min(abs((c + L) / h - round((c + L) / h)) for c in p) * h >= h / 4:
                    break
            nuc.append((tuple(p), 1.0))
        pk = [synth.packet([g.uniform(-4, 4) for _ in range(3)],
                           [g.uniform(-1.5, 1.5) for _ in range(3)])]
        specs.append(dict(nx=nx, nk=nk, nuclei=nuc, packets=pk,
                          nsteps=g.randint(steps[0], steps[1]),
                          precision=precisions[g.randint(0, len(precisions) - 1)],
                          L=L, lk=lk, dt=0.025))
    return specs


def run_serving(ch, n_req, rate, seed, nx_choices, nk_choices, steps, precisions, budget,
                max_slots, spl):
    """Submits the seeded stream with Poisson arrivals (rate per second) to the continuous-
    batching server and reports latency percentiles and aggregate cell-updates/s."""
    import synth
    specs = serving_specs(seed, n_req, nx_choices, nk_choices, steps, precisions)
    g = synth.SplitMix64(seed + 1)
    srv = ch.Server(budget, max_slots=max_slots, steps_per_launch=spl, queue_capacity=n_req)
    try:
        t0 = time.perf_counter()
        t_next = 0.0
        tickets = []
        for sp in specs:
            t_next += -math.log(1.0 - g.uniform()) / rate
            dly = t0 + t_next - time.perf_counter()
            if dly > 0:
                time.sleep(dly)
            req = ch.make_request(sp["nx"], sp["nk"], -sp["L"], sp["L"], sp["lk"], sp["dt"],
                                  sp["nsteps"], nuclei=sp["nuclei"], packets=sp["packets"],
                                  precision=sp["precision"])
            tickets.append(srv.submit(req))
        res = [srv.wait(t, 3600.0) for t in tickets]
        wall = time.perf_counter() - t0
    finally:
        srv.close()
    out = serving_stats([(sp["precision"], r.latency_ms, r.queue_ms, r.cells * r.nsteps, r.status)
                         for sp, r in zip(specs, res)], wall)
    out["rate_per_s"] = rate
    return out


def serving_both(ch, n_req, rate, steps, seed=2205, budget=150 << 30, max_slots=8, spl=5):
    """The same seeded request stream (grids {16,24,32}^3 x {16,32}^3, 1-2 protons, an electron
    packet, `steps` steps each, the same Poisson arrival times) served once in each form: the
    FP32-mixed form's latency percentiles next to the FP64 form's on the same GPU."""
    out = {}
    for name, prec in (("fp32_mixed", ch.FP32_MIXED), ("fp64", ch.FP64)):
        out[name] = run_serving(ch, n_req=n_req, rate=rate, seed=seed, nx_choices=(16, 24, 32),
                                nk_choices=(16, 32), steps=steps, precisions=(prec,),
                                budget=budget, max_slots=max_slots, spl=spl)
        r = out[name]
        r["mean_request_cell_updates"] = r["cell_updates_per_s"] * r["wall_s"] / n_req
    out["p99_ms_fp32_mixed_vs_fp64"] = [out["fp32_mixed"]["p99_ms"], out["fp64"]["p99_ms"]]
    out["sample"] = (f"{n_req} requests of the serving stream (grids {{16,24,32}}^3 x {{16,32}}^3, "
                     f"1-2 protons in [-2,2]^3, packet centre in [-4,4]^3, momentum in "
                     f"[-1.5,1.5]^3, {steps[0]}-{steps[1]} steps at dt 0.025, HBM budget 150 GB, "
                     f"{max_slots} slots), Poisson {rate}/s, the same stream in each form")
    return out


def latency_percentile(sorted_ms, q):
    """Nearest-rank percentile of an ascending list."""
    return sorted_ms[min(len(sorted_ms) - 1, max(0, int(math.ceil(q * len(sorted_ms))) - 1))]


def serving_stats(rows, wall):
    """Latency percentiles and throughput of a served stream from (precision, latency_ms,
    queue_ms, cell-updates, status) per request; with more than one precision in the stream also
    per precision (latencies of the requests of that precision in the same mixed run)."""
    def block(rs):
        lat = sorted(r[1] for r in rs)
        return {"requests": len(rs), "failed": sum(1 for r in rs if r[4] != 0),
                "p50_ms": latency_percentile(lat, 0.50), "p99_ms": latency_percentile(lat, 0.99),
                "mean_queue_ms": statistics.mean(r[2] for r in rs),
                "cell_updates": sum(r[3] for r in rs)}
    out = block(rows)
    out["cell_updates_per_s"] = out.pop("cell_updates") / wall
    out["wall_s"] = wall
    precs = sorted({r[0] for r in rows})
    if len(precs) > 1:
        names = {0: "fp32_mixed", 1: "fp64"}
        out["by_precision"] = {names.get(p, str(p)): block([r for r in rows if r[0] == p])
                               for p in precs}
    return out


def run_serve_mode(args):
    """The serving workload: 64 requests, grids {16,24,32}^3 x {16,32}^3, 10-100 steps, HBM budget
    150 GB, Poisson arrivals at --rate per second, in FP32-mixed; and the first
    --serve-fp64-requests requests of the same stream with at most 30 steps served in each form
    (the FP64 form runs on the FP64 pipe, about 30 times slower per cell on this GPU)."""
    import paper_2205_02380_gb300 as ch
    ch.chasm.lib()
    out = {"metric": "serving latency and throughput", "unit": "ms / cell-updates/s"}
    out["fp32_stream"] = run_serving(ch, n_req=args.serve_requests, rate=args.rate, seed=2205,
                                     nx_choices=(16, 24, 32), nk_choices=(16, 32),
                                     steps=(10, args.serve_max_steps), precisions=(ch.FP32_MIXED,),
                                     budget=150 << 30, max_slots=args.slots, spl=5)
    out["fp32_stream"]["sample"] = f"{args.serve_requests} requests, steps 10-{args.serve_max_steps}"
    if args.serve_fp64_requests > 0:
        out["both_forms"] = serving_both(ch, n_req=args.serve_fp64_requests, rate=args.fp64_rate,
                                         steps=(10, 30), max_slots=args.slots)
    print(json.dumps(out), flush=True)


def run_kernels(args):
    """Achieved bandwidth of the HBM-bound kernels outside the Strang step's pair (reductions,
    diagnostics, the quadratic-potential P-flow and Theta), FP32-mixed, on the full 32^3 x 32^3
    grid: algorithmic bytes per call / time per call.  Asynchronous calls are timed with CUDA
    events on the solver's stream; calls that return host values (they synchronise) by the wall
    clock around a synchronised loop, so their figure includes the call's return latency."""
    import torch
    import paper_2205_02380_gb300 as ch
    W = WORKLOADS[STATIONARITY]
    n, nk = W["nx"], W["nk"]
    fb = n ** 3 * nk ** 3 * 4
    peak = measured_hbm_gbs()
    stream = torch.cuda.Stream()
    res = {}

    def ev_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def wall_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps

    def put(name, kernels, ms, nbytes, how):
        gbs = nbytes / (ms / 1e3) / 1e9
        res[name] = {"kernels": kernels, "ms": ms, "algorithmic_bytes": nbytes, "gbs": gbs,
                     "frac_of_measured_hbm": (gbs / peak) if peak else None, "timing": how}

    shape = (n,) * 3 + (nk,) * 3
    with torch.cuda.stream(stream):
        s = make_solver(ch, W, ch.FP32_MIXED, stream)
        f = torch.empty(shape, device="cuda", dtype=torch.float32)
        init_f(s, W, f)
        put("mass_energy", "k_moments", wall_ms(lambda: s.moments(f), 5), fb, "wall")
        for j in range(3):
            put(f"reduced_wigner_{j}", "k_diag_kpart + k_diag_wigner",
                wall_ms(lambda: s.reduced_wigner(f, j), 3), fb, "wall")
        put("expectations", "3 x k_diag_kpart + k_diag_expect", wall_ms(lambda: s.expectations(f), 3),
            3 * fb, "wall")
        s.close()
        del f
        torch.cuda.empty_cache()
        h = ch.Solver(n, nk, -W["L"], W["L"], W["lk"], kappa=1.0, precision=ch.FP32_MIXED,
                      stream=stream.cuda_stream)
        f = torch.empty(shape, device="cuda", dtype=torch.float32)
        h.init_gaussians(f, [{"w": math.pi ** -3, "x0": (1.0, -0.5, 0.3), "k0": (0.5, 0.2, -0.4),
                              "ax": 0.5, "ak": 2.0}])
        put("harmonic_pflow", "3 x k_kshift", ev_ms(lambda: h.pflow(f, 1e-3), 5), 6 * fb, "events")
        out = torch.empty_like(f)
        put("harmonic_theta", "3 x k_kderiv", ev_ms(lambda: h.theta(f, out), 5), 8 * fb, "events")
        h.close()
    print(json.dumps({"kernels": res, "workload": "32^3 x 32^3 FP32 (f = %.1f GB)" % (fb / 1e9),
                      "peak_gbs": peak}))


def run_study_harmonic(args):
    """The 2-D phase-space harmonic oscillator of Sec. 5.1 through the 6-D solver: f = g(x1, k1)
    on the slice x2 = x3 = 0, k2 = k3 = 0 of 5-point x2, x3 grids, zero elsewhere (for a quadratic
    potential the step maps the product factor by factor and these unit factors are fixed points:
    no displacement along x_d at k_d = 0, no shift along k_d at x_d = 0), so the slice carries the
    (x1, k1) plane solution: V = kappa/2 x^2,
    kappa = (pi/5)^2 (period 10), f0 = pi^-1 exp(-(x1 - 1)^2/2 - 2 k1^2), x1 in [-12, 12] in 4
    PMBC patches, N_k = 32 on [-3.2, 3.2), FP64, Strang with dt = --study-dt over one period.
    After one period the exact solution is f0 again: eps_inf, eps_2 and eps_mass (Sec. 5) of the
    plane against f0, for a dx sweep at n_nb = 20 and an n_nb sweep at dx = 0.1."""
    import numpy as np
    import torch
    import paper_2205_02380_gb300 as ch
    kappa, T, lk, nk = (math.pi / 5) ** 2, 10.0, 3.2, 32
    dt = args.study_dt
    nsteps = int(round(T / dt))
    rows = []
    stream = torch.cuda.Stream()
    for nx, n_nb in ((81, 20), (121, 20), (241, 20), (241, 15), (241, 10)):
        h = 24.0 / (nx - 1)
        xs = -12.0 + h * np.arange(nx)
        ks = (np.arange(nk) - nk / 2) * (2 * lk / nk)
        X, K = np.meshgrid(xs, ks, indexing="ij")
        g0 = np.exp(-0.5 * (X - 1.0) ** 2 - 2.0 * K ** 2) / math.pi
        with torch.cuda.stream(stream):
            s = ch.Solver((nx, 5, 5), nk, (-12.0, -2.0, -2.0), (12.0, 2.0, 2.0), lk, nuclei=[],
                          kappa=kappa, precision=ch.FP64, n_nb=n_nb, patches=(4, 1, 1),
                          stream=stream.cuda_stream)
            f = torch.zeros((nx, 5, 5, nk, nk, nk), device="cuda", dtype=torch.float64)
            f[:, 2, 2, :, nk // 2, nk // 2] = torch.from_numpy(g0).to("cuda")
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step(f, dt, nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            g = f[:, 2, 2, :, nk // 2, nk // 2].cpu().numpy()
            f[:, 2, 2, :, nk // 2, nk // 2] = 0
            spread = float(f.abs().max())
            s.close()
            del f
            torch.cuda.empty_cache()
        d = g - g0
        cell = h * (2 * lk / nk)
        rows.append({"nx": nx, "dx": h, "n_nb": n_nb, "eps_inf": float(np.abs(d).max()),
                     "eps_2": float(np.sqrt((d * d).sum() * cell)),
                     "eps_mass": float(abs(d.sum()) * cell), "off_slice_max": spread,
                     "ms_per_step": e0.elapsed_time(e1) / nsteps})
    dxs = [r for r in rows if r["n_nb"] == 20]
    order = [math.log(a["eps_inf"] / b["eps_inf"]) / math.log(a["dx"] / b["dx"])
             for a, b in zip(dxs, dxs[1:])]
    print(json.dumps({"study": "harmonic oscillator, Sec. 5.1 (2-D phase space, 4 patches)",
                      "dt": dt, "steps": nsteps, "T": T, "rows": rows,
                      "order_eps_inf_dx": order}), flush=True)


def run_study_tkm(args):
    """Example 4.1 on the GPU: Phi = |k|^-2 * exp(-|k|^2) by chasm_tkm_convolve (the TKM of Sec. 4)
    for N_k = 8, 16, 32 on [-4, 4)^3, against the closed form 2 pi^{3/2} F(k)/k (F = Dawson's
    integral, scipy.special.dawsn): eps_inf = max |Phi - Phi_exact|, eps_2 = (sum (Phi -
    Phi_exact)^2 dk^3)^{1/2}, and the time per Phi (one x point) when 32^3 of them are computed in
    one call (CUDA events, mean of 5 calls), in both forms."""
    import numpy as np
    import torch
    from scipy.special import dawsn
    import paper_2205_02380_gb300 as ch
    lk, nx = 4.0, 32
    rows = []
    stream = torch.cuda.Stream()
    for prec, dtp, name in ((ch.FP64, torch.float64, "fp64"), (ch.FP32_MIXED, torch.float32, "fp32")):
        for nk in (8, 16, 32):
            dk = 2 * lk / nk
            ks = (np.arange(nk) - nk / 2) * dk
            K = np.sqrt(ks[:, None, None] ** 2 + ks[None, :, None] ** 2 + ks[None, None, :] ** 2)
            Kp = np.where(K > 0, K, 1.0)
            ex = np.where(K > 0, 2 * math.pi ** 1.5 * dawsn(Kp) / Kp, 2 * math.pi ** 1.5)
            with torch.cuda.stream(stream):
                s = ch.Solver(nx, nk, -12.0, 12.0, lk, nuclei=[((0.0, 0.0, 0.0), 1.0)],
                              theta_form=ch.THETA_TABLE, precision=prec, stream=stream.cuda_stream)
                g = torch.from_numpy(np.exp(-K ** 2)).to("cuda", dtp).expand(
                    (nx,) * 3 + (nk,) * 3).contiguous()
                out = torch.empty_like(g)
                s.tkm_convolve(g, out)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(5):
                    s.tkm_convolve(g, out)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / 5
                phi = out[0, 0, 0].double().cpu().numpy()
                s.close()
                del g, out
                torch.cuda.empty_cache()
            d = phi - ex
            rows.append({"form": name, "nk": nk, "eps_inf": float(np.abs(d).max()),
                         "eps_2": float(np.sqrt((d * d).sum() * dk ** 3)),
                         "s_per_phi": ms / 1e3 / nx ** 3, "ms_per_call": ms, "points": nx ** 3})
    print(json.dumps({"study": "Example 4.1 (TKM, Gaussian), L_k = 4", "rows": rows}), flush=True)


def run_long(args):
    """A full-length run of one workload in both forms from the same initial data (FP64 first; its
    result stays on the device while the FP32-mixed form runs): the relative L2 distance of the
    FP32-mixed result from the FP64 one, and per form the relative drift of mass and energy and
    the step time.  --long electron-proton runs its 100 steps (dt 0.02)."""
    import torch
    import paper_2205_02380_gb300 as ch
    W = WORKLOADS[args.long]
    steps = args.long_steps
    stream = torch.cuda.Stream()
    out, final = {}, None
    with torch.cuda.stream(stream):
        for name, prec, dtp in (("fp64", ch.FP64, torch.float64), ("fp32", ch.FP32_MIXED, torch.float32)):
            s = make_solver(ch, W, prec, stream)
            f = new_f(torch, W, dtp)
            init_f(s, W, f)
            m0, e0 = s.moments(f)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            s.step(f, W["dt"], steps)
            ev1.record(stream)
            torch.cuda.synchronize()
            m1, e1 = s.moments(f)
            out[name] = {"ms_per_step": ev0.elapsed_time(ev1) / steps, "mass_drift": (m1 - m0) / m0,
                         "energy0": e0, "energy_drift": (e1 - e0) / abs(e0)}
            s.close()
            if name == "fp64":
                final = f
            else:
                num = torch.linalg.vector_norm(f.double() - final)
                out["rel_l2_fp32_vs_fp64"] = float(num / torch.linalg.vector_norm(final))
                out["mass_rel_diff_fp32_vs_fp64"] = (out["fp32"]["mass_drift"] - out["fp64"]["mass_drift"])
            del f
            torch.cuda.empty_cache()
    print(json.dumps({"long_run": W["name"], "steps": steps, "t_final": steps * W["dt"],
                      "tolerance": 1e-5, **out}), flush=True)


def run_profile(args):
    """FP32 form only on --workload (default the headline one, --nx overrides N_x): init, W
    warm-up steps and K steps, nothing else (for ncu)."""
    import torch
    import paper_2205_02380_gb300 as ch
    W = WORKLOADS[args.workload]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = make_solver(ch, W, ch.FP32_MIXED, stream)
        f = new_f(torch, W, torch.float32)
        init_f(s, W, f)
        ms, _ = time_steps(torch, s, f, W["dt"], args.steps, args.warmup, stream, None)
        s.close()
    print(json.dumps({"profile_ms_per_step": ms / max(1, args.steps), "workload": W["name"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chasm", choices=["chasm", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--stat-steps", type=int, default=40,
                    help="steps of the hydrogen 1s stationarity run in both forms (0: skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true")
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(WORKLOADS))
    ap.add_argument("--profile", action="store_true",
                    help="FP32 timed steps only (no FP64, e2e, baseline or clocks): for ncu captures")
    ap.add_argument("--nx", type=int, default=None, help="override N_x (profiling on smaller cases)")
    ap.add_argument("--nk", type=int, default=None, help="override N_k (profiling on smaller cases)")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-lpc1", action="store_true")
    ap.add_argument("--bench-serve-requests", type=int, default=8)
    ap.add_argument("--bench-serve-rate", type=float, default=2.0)
    ap.add_argument("--kernels", action="store_true",
                    help="bandwidth of the reduction, diagnostic and quadratic-potential kernels")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--study", default="", choices=["", "harmonic", "tkm"],
                    help="harmonic: the Sec. 5.1 oscillator study (dx and n_nb sweeps); "
                         "tkm: the Example 4.1 table")
    ap.add_argument("--study-dt", type=float, default=0.005)
    ap.add_argument("--long", default="", choices=[""] + sorted(WORKLOADS),
                    help="full-length run of a workload in both forms (see --long-steps)")
    ap.add_argument("--long-steps", type=int, default=100)
    ap.add_argument("--rate", type=float, default=5.0)
    ap.add_argument("--fp64-rate", type=float, default=0.2)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-max-steps", type=int, default=100)
    ap.add_argument("--serve-fp64-requests", type=int, default=16)
    args = ap.parse_args()
    if args.nx:
        W = WORKLOADS[args.workload]
        old = f"{W['nx']}^3x"
        W["nx"] = args.nx
        W["name"] = W["name"].replace(old, f"{args.nx}^3x")
    if args.nk:
        W = WORKLOADS[args.workload]
        old = f"x{W['nk']}^3"
        W["nk"] = args.nk
        W["name"] = W["name"].replace(old, f"x{args.nk}^3")
    if args.profile:
        run_profile(args)
        return
    if args.kernels:
        run_kernels(args)
        return
    if args.serve:
        run_serve_mode(args)
        return
    if args.study == "harmonic":
        run_study_harmonic(args)
        return
    if args.study == "tkm":
        run_study_tkm(args)
        return
    if args.long:
        run_long(args)
        return
    if args.oracle_sample:
        print(json.dumps(cpu_baseline_run(args.workload)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_chasm(args)


if __name__ == "__main__":
    main()
