"""Benchmark: TEBD gate-updates/s at chi_max on one GB300 (and N replicas).

Workload (default): L=32 Bose-Hubbard chain with NN+NNN hopping and a trap
(U=5, J=1, J_NNN=0.12, K=0.005, j_c=16.5), d=4, chi_max=256, discarded-weight
cut 1e-10, dt=0.01, started from the seeded synthetic saturated state
(chi = min(256, 4^min(k, 32-k)) on every bond).  One step = one full
second-order Trotter step (A/2 B/2 C B/2 A/2 = 50 three-site gate updates,
100 truncated SVDs) plus the density/current measurement.  The state and
the workspace (> 2 GB) exceed L2 (129 MB), so no flush is needed between steps.

Multi-GPU: replicas only (independent simulations, one per rank, no
collective on the data path); value = all ranks' gate updates / max time.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (a few gate updates per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WL = workloads.TRUNC_L32
WORKLOADS = {"trunc_L32": workloads.TRUNC_L32, "parity_L8": workloads.PARITY_L8,
             "sample_L16_d5_chi1024": workloads.SAMPLE_L16_D5}


def gates_per_step(L: int) -> int:
    """Three-site gate updates in one A/2 B/2 C B/2 A/2 step (50 for L = 32)."""
    n = {r: len(range(r, L - 2, 3)) for r in range(3)}
    return 2 * n[0] + 2 * n[1] + n[2]


METRIC = "TEBD gate-updates/s at \u03c7_max, mixed vs FP64 on 1 GB300; served p50/p99 latency"
UNIT = "gate-updates/s"
# FP64 on GB300: 152 SMs x 2 DFMA (4 flop) per clock x 2070 MHz (a DFMA throughput
# probe measured 1.20 TFLOP/s at ~1970 MHz, i.e. 2 DFMA/clk/SM).
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# TF32 dense: measured bf16 peak x nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s).
TF32_RATIO = 1.1 / 2.25


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def config(precision: str):
    return {"workload": f"L{WL.L}_d{WL.d}_chi{WL.chi_max}_wcut{WL.w_cut:g}_synthetic_saturated",
            "L": WL.L, "d": WL.d, "chi_max": WL.chi_max, "dt": WL.dt, "precision": precision,
            "step": f"one 2nd-order Trotter step ({gates_per_step(WL.L)} three-site gate updates) + n_j/current measurement",
            "l2_flush": "not needed: state + workspace > 2 GB > 129 MB L2"}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 6:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest value of x over all ranks (the job's time is its slowest replica's)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def side_measurement(fn, *args):
    """Run a measurement reported beside the headline; if it fails, record why instead of losing the line."""
    try:
        return fn(*args)
    except Exception as e:
        return {"error": f"{type(e).__name__}: {e}"}


def job_value(updates_per_rank: int, ws: int, seconds_max: float) -> float:
    """Whole-job throughput of ws replicas that each did updates_per_rank gate updates."""
    return updates_per_rank * ws / seconds_max


def oracle_sample(n_gates: int, seed_state):
    """Time the oracle on n_gates three-site updates of the saturated state (layer A order)."""
    from oracle.tebd import TEBD as OracleTEBD
    B, lam, _ = seed_state
    o = OracleTEBD(WL.L, WL.n_max, WL.chi_max, WL.U, WL.J, WL.Jnnn, WL.K, WL.jc, WL.dt, w_cut=WL.w_cut,
                   eps_rel=WL.eps_rel)
    o.set_state(B, lam)
    triples = [j for j in range(1, WL.L - 1) if j % 3 == 1]
    gates = [o.gate(j, WL.dt / 2) for j in triples]  # built before timing (host setup, not the path)
    t0 = time.perf_counter()
    for q in range(n_gates):
        k = (q + 3) % len(triples)  # interior triples first
        o.apply_gate(triples[k] - 1, gates[k])
    return time.perf_counter() - t0


def served_requests(n: int = 24, rate: float = 8.0):
    """Seeded Poisson stream shaped like the serving workload, scaled to run in about a
    minute: 90% chains like the L=64, d=5 mixed-precision one (here L=24, chi_max=32,
    t = 0.2) and 10% larger d=4 jobs (L=40, chi_max=64, t = 0.4)."""
    from paper_2401_05301_gb300 import serving

    def make(i, t, rng):
        if rng.uniform() < 0.9:
            L = 24
            return serving.Request(rid=i, arrival=t, L=L, n_max=4, chi_max=32, U=3.0, J=1.0, Jnnn=0.1, K=0.003,
                                   jc=(L + 1) / 2, dt=0.005, n_steps=40, measure_every=10)
        L = 40
        return serving.Request(rid=i, arrival=t, L=L, n_max=3, chi_max=64, U=5.0, J=1.0, Jnnn=0.1, K=0.002,
                               jc=(L + 1) / 2, dt=0.01, n_steps=40, measure_every=10)

    return serving.poisson_requests(n, rate, workloads.SEED, make)


def served_measurement(stream_ptr):
    """Continuous batching (mixed path) vs one-at-a-time plain FP64 on the same stream."""
    from paper_2401_05301_gb300 import serving
    reqs = served_requests()
    srv = serving.Server(40e9, precision=1, stream_ptr=stream_ptr)
    batched = serving.latency_stats(srv.run(reqs))
    fifo_srv = serving.Server(40e9, precision=0, max_active=1, stream_ptr=stream_ptr)
    fifo = serving.latency_stats(fifo_srv.run(reqs))
    return {"requests": len(reqs), "arrival_rate_per_s": 8.0,
            "workload": "Poisson stream: 90% L=24 d=5 chi_max=32 t=0.2, 10% L=40 d=4 chi_max=64 t=0.4",
            "continuous_batching_mixed": batched, "one_at_a_time_fp64": fifo,
            "peak_active": srv.peak_active}


def batched_measurement(stream_ptr, steps: int = 10):
    """The 48 seeded simulations of the batched configuration (L in 16..64, chi_max in 64..512, d = 4),
    from their CDW product states: `tebd_batch_step` over all of them (one workspace slot each, so a
    layer's triples of many simulations share every grouped launch) against stepping each alone with
    its own default workspace.  Both start after one untimed step; mixed path."""
    import torch
    from paper_2401_05301_gb300 import TEBD, batch_step
    wls = workloads.batch48()

    def make(w, slots):
        g = TEBD(w.L, w.n_max, w.chi_max, w.U, w.J, w.Jnnn, w.K, w.jc, w.dt, precision=1, stream=stream_ptr)
        if slots:
            g.set_option("max_slots", slots)
        g.init_product(workloads.cdw(w.L))
        return g

    sims = [make(w, 1) for w in wls]
    batch_step(sims, 1)
    torch.cuda.synchronize()
    g0 = sum(g.counters()[0] for g in sims)
    t = time.perf_counter()
    batch_step(sims, steps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t
    gb = sum(g.counters()[0] for g in sims) - g0
    for g in sims:
        g.close()
    ta, ga = 0.0, 0
    for w in wls:
        g = make(w, 0)
        g.step(1)
        torch.cuda.synchronize()
        c0 = g.counters()[0]
        t = time.perf_counter()
        g.step(steps)
        torch.cuda.synchronize()
        ta += time.perf_counter() - t
        ga += g.counters()[0] - c0
        g.close()
    return {"workload": f"48 seeded simulations (L 16..64, chi_max 64..512, d=4) from CDW product states, "
                        f"{steps} steps after one untimed step", "unit": UNIT,
            "batched_value": gb / tb, "batched_s": tb, "alone_value": ga / ta, "alone_s": ta,
            "gate_updates": gb}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    state = workloads.synthetic_state(WL.L, WL.d, WL.chi_max)
    per_step = 2
    for _ in range(args.warmup):
        oracle_sample(per_step, state)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_sample(per_step, state)
    value = per_step * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config("fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{per_step} three-site updates of the saturated chi=256 state per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                    help="mixed: 3xTF32 tensor-core contractions + FP64 SVD (headline); the FP64 path is timed beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served p50/p99 measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-simulation batched measurement")
    ap.add_argument("--workload", default="trunc_L32", choices=sorted(WORKLOADS),
                    help="trunc_L32 is the measured configuration; parity_L8 is a small case for profiling")
    args = ap.parse_args()
    global WL
    WL = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    from paper_2401_05301_gb300 import TEBD

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    prec = 1 if args.precision == "mixed" else 0

    B, lam, chi = workloads.synthetic_state(WL.L, WL.d, WL.chi_max, seed=workloads.SEED + rank)
    g = TEBD(WL.L, WL.n_max, WL.chi_max, WL.U, WL.J, WL.Jnnn, WL.K, WL.jc, WL.dt, w_cut=WL.w_cut,
             eps_rel=WL.eps_rel, precision=prec, stream=stream.cuda_stream)
    g.set_state(B, lam)
    for _ in range(args.warmup):
        g.step(1)
        g.measure()

    def barrier():
        if ws > 1:
            dist.barrier()

    # -- device-timed region ------------------------------------------------------
    g.set_option("profile", 1)
    _, l0 = g.counters()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            g.step(1)
            g.measure()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    _, l1 = g.counters()
    prof = g.profile()
    g.set_option("profile", 0)
    t_max = max_over_ranks(ms, ws)
    value = job_value(gates_per_step(WL.L) * args.steps, ws, t_max / 1e3)

    # -- the plain FP64 path and the FP64-accurate tensor-core path on the same state ----
    def time_path(precision):
        gp = TEBD(WL.L, WL.n_max, WL.chi_max, WL.U, WL.J, WL.Jnnn, WL.K, WL.jc, WL.dt, w_cut=WL.w_cut,
                  eps_rel=WL.eps_rel, precision=precision, stream=stream.cuda_stream)
        gp.set_state(B, lam)
        for _ in range(args.warmup):
            gp.step(1)
            gp.measure()
        gp.set_option("profile", 1)
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            gp.step(1)
            gp.measure()
        f1.record(stream)
        torch.cuda.synchronize()
        fms = max_over_ranks(f0.elapsed_time(f1), ws)
        pp = gp.profile()
        gp.close()
        return {"value": job_value(gates_per_step(WL.L) * args.steps, ws, fms / 1e3), "unit": UNIT,
                "ms_per_step": fms / args.steps, "classes_ms": {k: round(v[0], 3) for k, v in pp.items()}}

    fp64 = exact = None
    if prec == 1:
        fp64 = time_path(0)
        exact = time_path(2)
        exact["note"] = ("precision 2: every large product on the exact-digit tensor-core engine "
                         "(FP64-accurate; parity with the oracle at the FP64 bound)")

    # -- end to end through the C ABI with host buffers ---------------------------
    pinned_B = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory().numpy() for b in B]
    pinned_l = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy() for x in lam]
    h2d = sum(b.nbytes for b in pinned_B) + sum(x.nbytes for x in pinned_l)
    d2h = 8 * (WL.L + WL.L - 1)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_state(pinned_B, pinned_l)
        g.step(1)
        g.measure()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e_value = job_value(gates_per_step(WL.L) * e2e_steps, ws, e2e_s)

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # -- roofline of the dominant kernel class ---------------------------------------
    dom = max((k for k in prof if k != "measure"), key=lambda k: prof[k][0])
    dms, dlaunch, dwork = prof[dom]
    achieved = dwork / (dms / 1e3) / 1e12 if dms > 0 else None
    roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
                "traffic": None,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 CUDA-core rate)",
                "share_of_step": dms / ms if ms > 0 else None,
                "classes_ms": {k: round(v[0], 3) for k, v in prof.items()},
                "classes_tflops": {k: (v[2] / (v[0] / 1e3) / 1e12 if v[0] > 0 and v[2] > 0 else None)
                                   for k, v in prof.items()}}

    if prec == 1 and prof["contract"][0] > 0:
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops")
        tf32_peak = bf16 * TF32_RATIO if bf16 else 1900.0 * TF32_RATIO
        tc_ach = prof["contract"][2] / (prof["contract"][0] / 1e3) / 1e12
        roofline["tensor_kernel"] = {
            "kernel": "k_tf32x3 (contract class)", "bound": "tensor", "achieved": tc_ach, "peak": tf32_peak,
            "unit": "TFLOP/s", "frac": tc_ach / tf32_peak, "traffic": None,
            "peak_source": ("measured bf16_tflops x 1.1/2.25 (nominal tf32/bf16)" if bf16 else
                            "fallback 1.9 PFLOP/s bf16 x 1.1/2.25"),
            "note": "algorithmic complex flops 8MNK; the 3xTF32 split issues 3x that on the tensor cores"}

    served = None
    if not args.no_served and ws == 1:
        served = side_measurement(served_measurement, stream.cuda_stream)
    batched = None
    if not args.no_batched and ws == 1 and args.workload == "trunc_L32":
        batched = side_measurement(batched_measurement, stream.cuda_stream)

    cpu = None
    if not args.no_cpu_baseline:
        n_cpu = 4
        secs = oracle_sample(n_cpu, (B, lam, chi))
        cpu = {"value": n_cpu / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n_cpu} three-site updates of the saturated chi=256 state ({secs:.1f} s)"}

    line = {"metric": METRIC,
            "metric_detail": ("value: mixed path (3xTF32 tensor-core contractions; SVD stage FP64-accurate, its "
                              "products as exact-digit tensor-core products); fp64_path: the plain FP64 GPU method on "
                              "the same state; exact_path: FP64-accurate throughout on the tensor cores"
                              if prec == 1 else "value: plain FP64 GPU method"),
            "value": value, "unit": UNIT, "svds_per_s": 2.0 * value, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f64+tf32x3",
            "data": "synthetic", "config": config(args.precision),
            "clocks": clk.summary(), "gpu_launches": int(l1 - l0),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h},
            "roofline": roofline, "cpu_baseline": cpu, "fp64_path": fp64, "exact_path": exact,
            "served": served, "batched": batched}
    print(json.dumps(line), flush=True)
    g.close()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
