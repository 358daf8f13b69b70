"""Benchmark: 6-D cell-updates per second of one Strang step of the CHASM scheme on GB300.

Workload (default): hydrogen 1s stationarity, V = -1/|x|, grid 32^3 x 32^3 on [-12,12]^3 x
[-4,4)^3 (1.07e9 cells), dt = 0.025, initial f = the 1s Wigner function (discrete Fourier sum,
N_y = 128) written on the GPU.  The headline `value` is the FP32-mixed form; the FP64 form is
measured on the same GPU and reported under "fp64".

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

WORKLOAD = {
    "name": "hydrogen-1s 32^3x32^3 [-12,12]^3 x [-4,4)^3, V=-1/|x|, dt=0.025",
    "nx": 32, "nk": 32, "L": 12.0, "lk": 4.0, "dt": 0.025,
    "nuclei": [((0.0, 0.0, 0.0), 1.0)], "n_y": 128,
}


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


def fp32_alu_peak_tflops() -> float:
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x the maximum SM clock."""
    mhz = 2070.0
    try:
        mhz = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        pass
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


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
    for name in ("k_theta_xs.cu", "fft_reg.cuh"):
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
def make_solver(ch, precision, stream, integrator=None):
    W = WORKLOAD
    return ch.Solver(W["nx"], W["nk"], -W["L"], W["L"], W["lk"], nuclei=W["nuclei"],
                     precision=precision, stream=stream.cuda_stream, theta_form=ch.THETA_TABLE,
                     integrator=ch.STRANG if integrator is None else integrator)


def time_lpc1(torch, ch, stream, steps, warmup):
    """The paper's LPC1 integrator on the same workload (FP32-mixed, table form): W untimed and
    `steps` timed steps, CUDA events on the solver's stream."""
    W = WORKLOAD
    with torch.cuda.stream(stream):
        s = make_solver(ch, ch.FP32_MIXED, stream, ch.LPC1)
        f = torch.empty((W["nx"],) * 3 + (W["nk"],) * 3, device="cuda", dtype=torch.float32)
        s.init_hydrogen_1s(f, n_y=W["n_y"])
        m0 = s.mass(f)
        ms = time_steps(torch, s, f, W["dt"], steps, warmup, stream, None)
        m1 = s.mass(f)
        s.close()
        del f
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    cells = W["nx"] ** 3 * W["nk"] ** 3
    return {"value": cells * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "dtype": "f32", "mass_drift": (m1 - m0) / m0,
            "note": "LPC1 (Sec. 2.2): 2 Theta applications and 6 advection passes per step (the "
                    "predictor and corrector base are formed inside the Theta kernel)"}


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
    """W untimed steps, then exactly `steps` Strang steps between CUDA events on the solver's
    stream, bracketed by barrier + synchronize.  Returns milliseconds."""
    s.step(f, dt, warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(f, dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


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


def cpu_baseline(seconds_target: float = 20.0):
    """Runs the FP64 oracle on a bounded sample of the workload in a fresh single-threaded
    process and returns its throughput (see oracle_sample)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample",
                        "--sample-seconds", str(seconds_target)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "failed: " + r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(seconds_target: float) -> dict:
    """Times the oracle's three substeps on pieces of the full-size workload:
    A(dt/2) on the full 32^3 x-cube at n_k sampled k points (the spline transform and the
    64-tap sum are independent per k), and P(dt) (four Theta^T applications) at n_x sampled x
    points (independent per x point).  Cell-update time = 2 t_A + t_P per cell."""
    import numpy as np

    import synth
    from oracle import chasm_oracle as O
    W = WORKLOAD
    nx, nk, L, lk, dt = W["nx"], W["nk"], W["L"], W["lk"], W["dt"]
    prob = O.Problem(nx=(nx,) * 3, nk=nk, x_lo=(-L,) * 3, x_hi=(L,) * 3, lk=lk,
                     nuclei=W["nuclei"])
    ks = prob.ks()
    # A: n_kA k points on the full x cube (surrogate smooth data; the cost is data independent)
    xs = prob.xs(0)
    g = np.exp(-0.5 * xs ** 2)
    n_kA = 2
    kidx = [(3, 17, 29), (20, 8, 14)][:n_kA]
    cube = (g[:, None, None] * g[None, :, None] * g[None, None, :])[..., None, None, None]
    t0 = time.perf_counter()
    for (a, b, c) in kidx:
        O.advect(cube, prob, 0.5 * dt, kaxes=(ks[a:a + 1], ks[b:b + 1], ks[c:c + 1]))
    tA = (time.perf_counter() - t0) / (n_kA * nx ** 3)
    # P: x points with the 1s data
    T = O.tkm_tensor(nk, lk)
    xpts = []
    tP_total, n_xP = 0.0, 0
    rng = np.random.default_rng(2205)
    while n_xP < 2 or tP_total < seconds_target * 0.5:
        i = rng.integers(0, nx, 3)
        x = np.array([xs[i[0]], xs[i[1]], xs[i[2]]])
        f1 = synth.wigner_1s((2, 2, 2), nk, tuple(x), tuple(x + 1.0), lk, n_y=W["n_y"])[:1, :1, :1]
        t0 = time.perf_counter()
        O.pflow_coulomb(f1.reshape(1, nk, nk, nk), prob, dt, T, xpts=x[None])
        tP_total += time.perf_counter() - t0
        n_xP += 1
        xpts.append(x)
        if n_xP >= 16:
            break
    tP = tP_total / (n_xP * nk ** 3)
    t_cell = 2 * tA + tP
    return {"value": 1.0 / t_cell, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle, 1 thread: A(dt/2) on the full 32^3 x-cube at {n_kA} "
                      f"k points ({tA * 1e6:.2f} us/cell) and P(dt) on {n_xP} x points of the 1s "
                      f"data ({tP * 1e6:.2f} us/cell); cell-update time = 2 t_A + t_P"}


# ------------------------------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = oracle_sample(max(2.0, 60.0 / max(1, args.steps + args.warmup)))
        if i >= args.warmup:
            per_step.append(r["value"])
    value = statistics.median(per_step)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "cells": WORKLOAD["nx"] ** 3 * WORKLOAD["nk"] ** 3,
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    W = WORKLOAD
    cells = W["nx"] ** 3 * W["nk"] ** 3
    dt = W["dt"]
    stream = torch.cuda.Stream()
    result = {}

    sampler = ClockSampler(local)
    for prec_name, prec, steps in (("fp32", ch.FP32_MIXED, args.steps),
                                   ("fp64", ch.FP64, max(1, min(args.steps, args.fp64_steps)))):
        with torch.cuda.stream(stream):
            s = make_solver(ch, prec, stream)
            dtp = torch.float32 if prec == ch.FP32_MIXED else torch.float64
            f = torch.empty((W["nx"],) * 3 + (W["nk"],) * 3, device="cuda", dtype=dtp)
            s.init_hydrogen_1s(f, n_y=W["n_y"])
            m0, e0 = s.moments(f)
            if prec_name == "fp32":
                sampler.start()
            ms = time_steps(torch, s, f, dt, steps, args.warmup if prec_name == "fp32" else 1,
                            stream, dist)
            if prec_name == "fp32":
                clocks = sampler.stop()
            m1, e1 = s.moments(f)
            ms_t, value = aggregate_ranks(ms, cells, steps, dist, "cuda")
            entry = {"ms_per_step": ms_t / steps, "steps": steps, "value": value,
                     "mass0": m0, "mass": m1, "energy0": e0, "energy": e1}
            entry["pflow_ms"] = time_pflow_launches(torch, s, f, dt, stream,
                                                    5 if prec_name == "fp32" else 1)
            if prec_name == "fp32":
                # end-to-end through the C ABI with HOST buffers (pinned), copies included
                host = torch.empty(f.shape, dtype=dtp, pin_memory=True)
                host.copy_(f)
                hout = torch.empty_like(host, pin_memory=True)
                k_e2e = max(1, min(steps, args.e2e_steps))
                s.run_host(host.data_ptr(), hout.data_ptr(), dt, 1)   # warm: buffer + graph
                runs = []
                for _ in range(3):   # median of three calls (host-side timing noise)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    s.run_host(host.data_ptr(), hout.data_ptr(), dt, k_e2e)
                    runs.append(time.perf_counter() - t0)
                t_e2e = statistics.median(runs)
                entry["e2e"] = {"value": world * cells * k_e2e / t_e2e, "unit": UNIT,
                                "h2d_bytes_per_step": s.f_bytes() / k_e2e,
                                "d2h_bytes_per_step": (s.f_bytes() + 8) / k_e2e,
                                "steps": k_e2e, "wall_s": t_e2e,
                                "host_copy_gbs": host_copy_gbs(torch, host, f, stream)}
                del host, hout
            del f
            s.close()
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        result[prec_name] = entry

    accuracy = accuracy_check(torch, ch, stream, args.acc_steps) if rank == 0 else None
    # the host-core baseline runs after the GPU measurements: its large host allocations, made
    # before the pinned e2e buffers, slowed the host <-> device copies of the e2e call (the child
    # process shares no CUDA state)
    base = cpu_baseline() if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    lpc1 = time_lpc1(torch, ch, stream, max(1, args.steps), 1) if rank == 0 and not args.no_lpc1 else None
    serving = None
    if rank == 0 and not args.no_serving:
        serving = run_serving(ch, n_req=16, rate=20.0, seed=2205, nx_choices=(16, 24),
                              nk_choices=(16,), steps=(10, 30), precisions=(ch.FP32_MIXED,),
                              budget=150 << 30, max_slots=8, spl=5)
        serving["sample"] = ("16 requests, Poisson 20/s, nx in {16,24}, nk 16, 10-30 steps, "
                             "FP32-mixed (the full 64-request stream: bench.py --serve)")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    r32, r64 = result["fp32"], result["fp64"]
    nk = W["nk"]
    flops_launch = 4 * theta_flops_per_cell(nk) * cells
    achieved = flops_launch / (r32["pflow_ms"] / 1e3) / 1e12
    achieved64 = flops_launch / (r64["pflow_ms"] / 1e3) / 1e12
    peak = fp32_alu_peak_tflops()
    try:
        fma32, fma64 = ch.chasm.fma_peaks()
        fma32x2 = ch.chasm.fma_peak_f32x2()
    except Exception:
        fma32 = fma64 = fma32x2 = None
    tr = committed_traffic()
    line = {
        "metric": METRIC, "value": r32["value"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r32["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (hydrogen 1s Wigner function computed on the GPU)",
        "config": {"workload": W["name"], "cells": cells, "global_batch": world,
                   "parallelism": f"replicas{world}",
                   "l2": "inputs larger than L2 (f = %.1f GB)" % (cells * 4 / 1e9)},
        "fp64": {"value": r64["value"], "ms_per_step": r64["ms_per_step"], "steps": r64["steps"],
                 "dtype": "f64", "pflow_ms": r64["pflow_ms"], "pflow_tflops": achieved64,
                 "pflow_frac_of_measured_fp64_fma": (achieved64 / fma64) if fma64 else None},
        "accuracy": accuracy,
        "lpc1": lpc1,
        "serving": serving,
        "roofline": {"kernel": "k_theta_xs (P(dt): four Horner stages of Theta^T per x point, "
                               "table form)",
                     "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock",
                     "measured_fma_peak_tflops": fma32,
                     "frac_of_measured_fma_peak": (achieved / fma32) if fma32 else None,
                     "measured_packed_f32x2_fma_tflops": fma32x2,
                     "ms_per_launch": r32["pflow_ms"],
                     "flops_per_launch": flops_launch,
                     "traffic": (tr["dram_bytes_per_launch"] * cells / tr["cells"]) if tr else None},
        "e2e": r32["e2e"],
        "gpu_launches": 7 * args.steps,
        "clocks": clocks,
        "cpu_baseline": base,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def accuracy_check(torch, ch, stream, steps):
    """Both forms from the same 1s initial data for `steps` steps: relative L2 of the FP32-mixed
    result against the FP64 result (the FP64 form is itself pinned to the FP64 oracle) and the
    relative mass drift of each."""
    W = WORKLOAD
    out = {}
    with torch.cuda.stream(stream):
        for name, prec, dtp in (("fp64", ch.FP64, torch.float64), ("fp32", ch.FP32_MIXED, torch.float32)):
            s = make_solver(ch, prec, stream)
            f = torch.empty((W["nx"],) * 3 + (W["nk"],) * 3, device="cuda", dtype=dtp)
            s.init_hydrogen_1s(f, n_y=W["n_y"])
            m0, _ = s.moments(f)
            s.step(f, W["dt"], steps)
            m1, _ = s.moments(f)
            out[name] = (f, (m1 - m0) / m0, m1)
            s.close()
        a, b = out["fp32"][0].double(), out["fp64"][0]
        rel = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
        res = {"steps": steps, "rel_l2_fp32_vs_fp64": rel, "tolerance": 1e-5,
               "mass_rel_diff_fp32_vs_fp64": (out["fp32"][2] - out["fp64"][2]) / out["fp64"][2],
               "mass_drift_fp32": out["fp32"][1], "mass_drift_fp64": out["fp64"][1],
               "note": "the FP64 form is pinned to the FP64 oracle at <= 1e-12"}
        del a, b, out
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


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
    150 GB, Poisson arrivals at --rate per second, in FP32-mixed.  The FP64 form runs on the FP64
    pipe (1/64 of the FP32 rate on this GPU; about 1.9 s per 32^3 x 32^3 step), so the stream
    that mixes both precisions is a bounded sample: --serve-mixed-requests requests (default 16)
    with at most 30 steps each."""
    import torch
    import paper_2205_02380_gb300 as ch
    ch.chasm.lib()
    out = {"metric": "serving latency and throughput", "unit": "ms / cell-updates/s"}
    plan = (("fp32", (ch.FP32_MIXED,), args.serve_requests, args.serve_max_steps),
            ("mixed", (ch.FP32_MIXED, ch.FP64), args.serve_mixed_requests, 30))
    for name, precs, n_req, max_steps in plan:
        if args.serve_precisions and name not in args.serve_precisions.split(","):
            continue
        out[name] = run_serving(ch, n_req=n_req, rate=args.rate, seed=2205,
                                nx_choices=(16, 24, 32), nk_choices=(16, 32),
                                steps=(10, max_steps), precisions=precs,
                                budget=150 << 30, max_slots=args.slots, spl=5)
        out[name]["sample"] = f"{n_req} requests, steps 10-{max_steps}"
    print(json.dumps(out), flush=True)


def run_kernels(args):
    """Achieved bandwidth of the HBM-bound kernels outside the Strang step's pair (reductions,
    diagnostics, the quadratic-potential P-flow and Theta), FP32-mixed, on the full 32^3 x 32^3
    grid: algorithmic bytes per call / time per call.  Asynchronous calls are timed with CUDA
    events on the solver's stream; calls that return host values (they synchronise) by the wall
    clock around a synchronised loop, so their figure includes the call's return latency."""
    import torch
    import paper_2205_02380_gb300 as ch
    W = WORKLOAD
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
        s = make_solver(ch, ch.FP32_MIXED, stream)
        f = torch.empty(shape, device="cuda", dtype=torch.float32)
        s.init_hydrogen_1s(f, n_y=W["n_y"])
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


def run_profile(args):
    """FP32 form only: init, W warm-up steps and K steps, nothing else (for ncu)."""
    import torch
    import paper_2205_02380_gb300 as ch
    W = WORKLOAD
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = make_solver(ch, ch.FP32_MIXED, stream)
        f = torch.empty((W["nx"],) * 3 + (W["nk"],) * 3, device="cuda", dtype=torch.float32)
        s.init_hydrogen_1s(f, n_y=W["n_y"])
        ms = time_steps(torch, s, f, W["dt"], args.steps, args.warmup, stream, None)
        s.close()
    print(json.dumps({"profile_ms_per_step": ms / max(1, args.steps), "nx": W["nx"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="chasm", choices=["chasm", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="FP32 timed steps only (no FP64, e2e, baseline or clocks): for ncu captures")
    ap.add_argument("--nx", type=int, default=None, help="override N_x (profiling on smaller cases)")
    ap.add_argument("--acc-steps", type=int, default=4)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-lpc1", action="store_true")
    ap.add_argument("--kernels", action="store_true",
                    help="bandwidth of the reduction, diagnostic and quadratic-potential kernels")
    ap.add_argument("--serve", action="store_true", help="run the serving workload instead")
    ap.add_argument("--rate", type=float, default=5.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-max-steps", type=int, default=100)
    ap.add_argument("--serve-mixed-requests", type=int, default=16)
    ap.add_argument("--serve-precisions", default="")
    ap.add_argument("--sample-seconds", type=float, default=20.0)
    args = ap.parse_args()
    if args.nx:
        WORKLOAD["nx"] = args.nx
        WORKLOAD["name"] = WORKLOAD["name"].replace("32^3x32^3", f"{args.nx}^3x32^3")
    if args.profile:
        run_profile(args)
        return
    if args.kernels:
        run_kernels(args)
        return
    if args.serve:
        run_serve_mode(args)
        return
    if args.oracle_sample:
        print(json.dumps(oracle_sample(args.sample_seconds)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_chasm(args)


if __name__ == "__main__":
    main()
