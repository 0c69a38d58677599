"""Benchmark: TEBD gate-updates/s at chi_max on one GB300 (and N replicas).

Workload (default, "L64_d5_chi1024_u1"): the mixed-precision chain of L = 64 sites,
n_max = 4 (d = 5), U = 3, J = 1, J_NNN = 0.1, K = 0.003 about j_c = 32.5,
dt = 0.005, chi_max = 1024, relative cut eps = 1e-12, at half filling
(N = 32), started from the seeded charge-labelled synthetic saturated state
(chi_k = min(1024, 5^min(k, 64-k)): bonds 5..59 at chi_max = 1024; right-
canonical charge blocks; lambda with p_i ~ exp(-8 i / chi)).  One step = one
full second-order Trotter step (A/2 B/2 C B/2 A/2 = 104 three-site gate
updates, 208 truncated SVDs) plus the density/current measurement, on the
particle-number-blocked form of the update (the paper's U(1)-symmetric
decompositions, Sec. II B).  The state (5.4 GB) and workspace exceed L2
(129 MB), so no flush is needed between steps.

value: the mixed path (3xTF32 tensor-core contractions, FP64-accurate
decompositions).  Beside it: the plain FP64 path and the FP64-accurate
exact-digit path on the same state (a stated number of steps each), and the
dense form on the L = 32, d = 4, chi = 256 chain.

Multi-GPU: replicas only (independent simulations, one per rank, no
collective on the data path); value = all ranks' gate updates / max time.

--impl reference times the CPU oracle on the host cores on a bounded sample
of the same workload (see run_reference).
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

HEAD = workloads.MIXED_L64
N_HEAD = 32              # bosons of the 64-site half-filled CDW
SIDE_STEPS = 3           # timed steps of the FP64 and exact-digit side arms
REF_CHI = 384           # chi_max of the reference arm's CPU sample (see run_reference)

METRIC = "TEBD gate-updates/s at χ_max, mixed vs FP64 on 1 GB300; served p50/p99 latency"
UNIT = "gate-updates/s"
# FP64 on GB300: 152 SMs x 2 DFMA (4 flop) per clock x 2070 MHz (a DFMA throughput
# probe measured 1.20 TFLOP/s at ~1970 MHz, i.e. 2 DFMA/clk/SM).
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# TF32 dense: measured bf16 peak x nominal tf32/bf16 ratio (1.1 / 2.25 PFLOP/s).
TF32_RATIO = 1.1 / 2.25
ALU_CLASSES = ("tridiag", "bisect", "eigvec")


def gates_per_step(L: int) -> int:
    """Three-site gate updates in one A/2 B/2 C B/2 A/2 step (104 for L = 64, 50 for L = 32)."""
    n = {r: len(range(r, L - 2, 3)) for r in range(3)}
    return 2 * n[0] + 2 * n[1] + n[2]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def blas_vendor() -> str:
    try:
        b = np.__config__.CONFIG["Build Dependencies"]["blas"]
        return f"{b.get('name')} {b.get('version')}"
    except Exception:  # noqa: BLE001 - a description only
        return "unknown"


def head_config(precision: str):
    wl = HEAD
    return {"workload": f"L{wl.L}_d{wl.d}_chi{wl.chi_max}_N{N_HEAD}_u1_synthetic_saturated",
            "L": wl.L, "d": wl.d, "chi_max": wl.chi_max, "N": N_HEAD, "U": wl.U, "J": wl.J, "J_NNN": wl.Jnnn,
            "K": wl.K, "j_c": wl.jc, "dt": wl.dt, "eps_rel": wl.eps_rel, "w_cut": wl.w_cut, "precision": precision,
            "form": "particle-number (U(1)) blocked local update, dense site tensors in HBM",
            "step": f"one 2nd-order Trotter step ({gates_per_step(wl.L)} three-site gate updates) + n_j/current "
                    "measurement",
            "l2_flush": "not needed: state (5.4 GB) + workspace > 129 MB L2"}


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


PANEL_LAUNCH_DRAM_BYTES = 41.27e6  # 38.92 MB read + 2.35 MB written (ncu, the current kernel)


def side_measurement(fn, *args, **kw):
    """Run a measurement reported beside the headline; if it fails, record why instead of losing the line."""
    try:
        return fn(*args, **kw)
    except Exception as e:  # noqa: BLE001 - reported, not swallowed
        return {"error": f"{type(e).__name__}: {e}"}


def job_value(updates_per_rank: int, ws: int, seconds_max: float) -> float:
    """Whole-job throughput of ws replicas that each did updates_per_rank gate updates."""
    return updates_per_rank * ws / seconds_max


def head_state(seed: int = workloads.SEED, chi_max: int = HEAD.chi_max):
    return workloads.synthetic_state_u1(HEAD.L, HEAD.d, chi_max, N_HEAD, seed=seed)


def oracle_update_seconds(state, chi_max: int = HEAD.chi_max, n: int = 1) -> float:
    """Time the U(1) oracle on n gate updates of the interior triple on sites 31..33 of the
    charge-labelled saturated chain (the gate is built before the clock starts)."""
    from oracle.u1 import U1TEBD
    B, lam, q = state
    o = U1TEBD(HEAD.L, HEAD.n_max, chi_max, HEAD.U, HEAD.J, HEAD.Jnnn, HEAD.K, HEAD.jc, HEAD.dt,
               w_cut=HEAD.w_cut, eps_rel=HEAD.eps_rel)
    total = 0.0
    j = HEAD.L // 2 - 1  # the interior triple (sites 31..33 of the 64-site chain)
    G = o.gate(j, HEAD.dt / 2)
    for _ in range(n):
        o.set_state(B, lam, q)
        t0 = time.perf_counter()
        o.apply_gate(j - 1, G)
        total += time.perf_counter() - t0
    return total


def profile_summary(prof):
    return {"classes_ms": {k: round(v[0], 3) for k, v in prof.items()},
            "classes_tflops": {k: (v[2] / (v[0] / 1e3) / 1e12 if v[0] > 0 and v[2] > 0 else None)
                               for k, v in prof.items()}}


def make_head(precision: int, stream_ptr: int, state):
    from paper_2401_05301_gb300 import TEBD
    wl = HEAD
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut,
             eps_rel=wl.eps_rel, precision=precision, stream=stream_ptr, u1=True)
    B, lam, q = state
    g.set_state(B, lam)
    g.set_charges(q)
    return g


def time_path(precision: int, state, stream, steps: int, warmup: int, ws: int, barrier):
    """A side arm on the headline state: warmup + steps full steps, device-timed."""
    import torch
    g = make_head(precision, stream.cuda_stream, state)
    for _ in range(warmup):
        g.step(1)
        g.measure()
    g.set_option("profile", 1)
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(steps):
        g.step(1)
        g.measure()
    f1.record(stream)
    torch.cuda.synchronize()
    fms = max_over_ranks(f0.elapsed_time(f1), ws)
    pp = g.profile()
    g.close()
    out = {"value": job_value(gates_per_step(HEAD.L) * steps, ws, fms / 1e3), "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": fms / steps}
    out.update(profile_summary(pp))
    return out


def dense_L32(stream, steps: int = 2, warmup: int = 1):
    """The dense form on the L = 32, d = 4, chi = 256 chain (w_cut = 1e-10) from its seeded
    synthetic saturated state: mixed, plain FP64 and exact-digit paths."""
    import torch
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.TRUNC_L32
    B, lam, _ = workloads.synthetic_state(wl.L, wl.d, wl.chi_max)
    out = {"workload": f"L{wl.L}_d{wl.d}_chi{wl.chi_max}_wcut{wl.w_cut:g}_synthetic_saturated (dense form)",
           "steps": steps, "warmup": warmup}
    for name, prec in (("mixed", 1), ("fp64", 0), ("exact", 2)):
        g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut,
                 eps_rel=wl.eps_rel, precision=prec, stream=stream.cuda_stream)
        g.set_state(B, lam)
        for _ in range(warmup):
            g.step(1)
        g.set_option("profile", 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.step(1)
            g.measure()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        prof = g.profile()
        g.close()
        tri = prof["tridiag"]
        out[name] = {"value": gates_per_step(wl.L) * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
                     "tridiag_frac_of_fp64_peak": (tri[2] / (tri[0] / 1e3) / 1e12 / FP64_PEAK_TFLOPS
                                                   if tri[0] > 0 else None)}
        out[name].update(profile_summary(prof))
    return out


SERVE_REQUESTS = 16      # the served mix is 500 requests; scaled to fit a bounded run
SERVE_STEPS = (12, 6)    # steps of the headline-style / large requests (unscaled: to t = 8 / t = 6)
SERVE_SLOTS = 4          # workspace slots per request (more requests fit the budget)
SERVE_CONCURRENT = 6     # the HBM budget admits about this many headline-style requests at once


def serve_stream(rate: float, seed: int = workloads.SEED, n: int = SERVE_REQUESTS, blocked: bool = True,
                 at_once: bool = False):
    """The served request mix, scaled: 90% chains like the headline (L=64, d=5, chi_max=1024, U=3,
    J_NNN=0.1, K=0.003 about j_c=32.5, dt=0.005) and 10% large jobs (L=100, d=4, chi_max=2048, U=5,
    J_NNN=0.1, K=0.002 about j_c=50.5, dt=0.01), each from its CDW state, measured every 4 steps.
    Seeded draws: the exponential inter-arrival times first, then the request types."""
    from paper_2401_05301_gb300 import serving
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n) if rate > 0 else np.zeros(n)
    large = rng.uniform(size=n) >= 0.9
    out, t = [], 0.0
    for i in range(n):
        t = 0.0 if at_once else t + float(gaps[i])
        if large[i]:
            L = 100
            out.append(serving.Request(rid=i, arrival=t, L=L, n_max=3, chi_max=2048, U=5.0, J=1.0, Jnnn=0.1,
                                       K=0.002, jc=(L + 1) / 2, dt=0.01, n_steps=SERVE_STEPS[1], measure_every=4,
                                       max_slots=SERVE_SLOTS, u1=blocked))
        else:
            wl = HEAD
            out.append(serving.Request(rid=i, arrival=t, L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U,
                                       J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc, dt=wl.dt, n_steps=SERVE_STEPS[0],
                                       measure_every=4, max_slots=SERVE_SLOTS, u1=blocked))
    return out


def served_measurement(stream_ptr):
    """Continuous batching of the blocked mixed-precision form under an HBM budget that admits
    about SERVE_CONCURRENT headline-style requests at once, against one-at-a-time plain FP64
    (the dense form, precision 0) on the same stream.  Capacity = requests/s with every request
    waiting at t = 0; the Poisson streams then offer 0.5, 0.9 and 1.2 of it."""
    from paper_2401_05301_gb300 import binding, serving
    small = binding.estimate_bytes(HEAD.L, HEAD.n_max, HEAD.chi_max, SERVE_SLOTS, 1, u1=True)
    large = binding.estimate_bytes(100, 3, 2048, SERVE_SLOTS, 1, u1=True)
    budget = max(SERVE_CONCURRENT * small, 1.05 * large)

    def serve(reqs, precision=1, max_active=64, hbm=budget):
        srv = serving.Server(hbm, precision=precision, max_active=max_active, stream_ptr=stream_ptr)
        t0 = time.perf_counter()
        res = srv.run(reqs)
        return serving.latency_stats(res), time.perf_counter() - t0, srv

    cap_stats, cap_s, _ = serve(serve_stream(0.0, at_once=True))
    capacity = SERVE_REQUESTS / cap_s
    loads = {}
    for load in (0.5, 0.9, 1.2):
        st, wall, srv = serve(serve_stream(load * capacity))
        st["peak_active"] = srv.peak_active
        st["peak_budget_fraction"] = srv.peak_used / budget
        loads[f"{load:g}"] = st
    fifo_stats, fifo_s, _ = serve(serve_stream(0.9 * capacity, blocked=False), precision=0, max_active=1,
                                  hbm=float("inf"))
    return {"workload": (f"served mix scaled: {SERVE_REQUESTS} Poisson requests (500 unscaled), 90% "
                         f"L=64 d=5 chi_max=1024 for {SERVE_STEPS[0]} steps (t=8 unscaled), 10% L=100 d=4 "
                         f"chi_max=2048 for {SERVE_STEPS[1]} steps (t=6), each from its CDW state, "
                         f"{SERVE_SLOTS} workspace slots per request"),
            "hbm_budget_bytes": budget, "footprint_bytes": {"headline_style": small, "large": large},
            "capacity_requests_per_s": capacity, "capacity_run": cap_stats,
            "continuous_batching_mixed_blocked": loads,
            "one_at_a_time_fp64_dense_at_0.9": {**fifo_stats, "wall_s": fifo_s}}


def batched_measurement(stream_ptr, steps: int = 1):
    """The 48-simulation batch: seeded simulations (L in 16..64, chi_max in 64..512, d = 4, seeded U, J_NNN,
    K; j_c = (L+1)/2), warm-started at chi_max: each from the charge-labelled synthetic saturated
    state of its chain at half filling (N = L/2), blocked form, mixed precision.  One
    `tebd_batch_step` over all 48 (every stage of a layer is one grouped launch over the triples of
    many simulations) against stepping each alone; both after one untimed step."""
    import torch
    from paper_2401_05301_gb300 import TEBD, batch_step
    wls = workloads.batch48()
    states = [workloads.synthetic_state_u1(w.L, w.d, w.chi_max, w.L // 2, seed=workloads.SEED + 1000 + i)
              for i, w in enumerate(wls)]

    def make(w, st):
        g = TEBD(w.L, w.n_max, w.chi_max, w.U, w.J, w.Jnnn, w.K, w.jc, w.dt, precision=1, stream=stream_ptr,
                 u1=True)
        B, lam, q = st
        g.set_state(B, lam)
        g.set_charges(q)
        return g

    sims = [make(w, st) for w, st in zip(wls, states)]
    batch_step(sims, 1)
    torch.cuda.synchronize()
    g0 = sum(g.counters()[0] for g in sims)
    l0 = sims[0].counters()[1]
    t = time.perf_counter()
    batch_step(sims, steps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t
    gb = sum(g.counters()[0] for g in sims) - g0
    lb = sims[0].counters()[1] - l0  # the first handle drives the batch and counts its launches
    for g in sims:
        g.close()
    ta, ga, la = 0.0, 0, 0
    for w, st in zip(wls, states):
        g = make(w, st)
        g.step(1)
        torch.cuda.synchronize()
        c0, k0 = g.counters()
        t = time.perf_counter()
        g.step(steps)
        torch.cuda.synchronize()
        ta += time.perf_counter() - t
        c1, k1 = g.counters()
        ga += c1 - c0
        la += k1 - k0
        g.close()
    return {"workload": f"48 seeded simulations (L 16..64, chi_max 64..512, d=4, N=L/2) from their "
                        f"charge-labelled synthetic saturated states, {steps} steps after one untimed step, "
                        f"blocked form, mixed precision", "unit": UNIT,
            "batched_value": gb / tb, "batched_s": tb, "alone_value": ga / ta, "alone_s": ta,
            "gate_updates": gb, "launches_per_step_batched": lb / steps, "launches_per_step_alone": la / steps,
            "speedup": (gb / tb) / (ga / ta)}


def graph_measurement(stream_ptr, steps: int = 6):
    """Launch-bound dense steps with and without CUDA-graph replay (option "graph"): the
    first 16 of the 48-simulation batch's draws (L 16..64, d = 4) at chi_max capped to 64, each from
    its dense synthetic saturated state, mixed precision, one batch.  Both arms run two untimed
    steps first (with the option on: one ordinary, one captured), then `steps` timed steps."""
    import torch
    from paper_2401_05301_gb300 import TEBD, batch_step
    wls = workloads.batch48()[:16]

    def arm(graph):
        sims = []
        for i, w in enumerate(wls):
            chi = min(w.chi_max, 64)
            g = TEBD(w.L, w.n_max, chi, w.U, w.J, w.Jnnn, w.K, w.jc, w.dt, precision=1, stream=stream_ptr)
            B, lam, _ = workloads.synthetic_state(w.L, w.d, chi, seed=workloads.SEED + 2000 + i)
            g.set_state(B, lam)
            if graph:
                g.set_option("graph", 1)
            sims.append(g)
        batch_step(sims, 2)
        torch.cuda.synchronize()
        g0 = sum(g.counters()[0] for g in sims)
        l0 = sims[0].counters()[1]
        t = time.perf_counter()
        batch_step(sims, steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        gu = sum(g.counters()[0] for g in sims) - g0
        launches = sims[0].counters()[1] - l0
        stats = sims[0].graph_stats()
        for g in sims:
            g.close()
        return {"value": gu / dt, "seconds": dt, "gate_updates": gu, "kernels_per_step": launches / steps,
                "graph_replays": stats[0], "graph_fallbacks": stats[1]}

    plain = arm(False)
    graph = arm(True)
    return {"workload": f"16 seeded simulations (the 48-batch's first draws, L 16..64, d=4, chi_max capped at 64) from dense "
                        f"synthetic saturated states, one batch, mixed precision, {steps} steps after two untimed",
            "unit": UNIT, "ordinary": plain, "graph": graph, "speedup": graph["value"] / plain["value"]}


def run_reference(args):
    """The CPU oracle (oracle/u1.py, numpy + LAPACK FP64, the machine's host cores) on the headline
    chain's physics.  One oracle update of a saturated triple at chi_max = 1024 takes ~50 s on 8
    x86 host cores (measured), so no bounded run of --steps K full-size updates fits in minutes;
    each step here is one update of the same interior triple of the same charge-labelled chain
    with chi_max = REF_CHI (the cost grows as chi^3)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    state = head_state(chi_max=REF_CHI)
    for _ in range(args.warmup):
        oracle_update_seconds(state, REF_CHI)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_update_seconds(state, REF_CHI)
    value = args.steps / total
    cfg = head_config("fp64")
    cfg["cpu_sample_chi_max"] = REF_CHI
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "blas": blas_vendor(),
                             "kind": "oracle",
                             "sample": f"one U(1)-oracle gate update per step, interior triple of the L=64 d=5 "
                                       f"charge-labelled saturated chain at chi_max={REF_CHI} (1024 does not fit "
                                       f"a bounded run)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_dense_workload(args):
    """--workload trunc_L32: the dense form on the L = 32, d = 4, chi = 256 chain alone."""
    import torch
    torch.cuda.set_device(0)
    out = dense_L32(torch.cuda.current_stream(), steps=args.steps, warmup=args.warmup)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="L64_d5_chi1024_u1", choices=["L64_d5_chi1024_u1", "u1_L24", "trunc_L32"],
                    help="L64_d5_chi1024_u1: the headline (L=64 d=5 chi=1024, blocked form); u1_L24: the same physics and "
                         "local sizes on 24 sites (N=12; a small case for profiling); trunc_L32: the dense form alone")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-served", action="store_true", help="skip the served p50/p99 measurement")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-simulation batched measurement")
    ap.add_argument("--no-side", action="store_true", help="skip the FP64 / exact-digit / dense side arms")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay measurement")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "trunc_L32":
        return run_dense_workload(args)
    if args.workload == "u1_L24":
        global HEAD, N_HEAD
        HEAD = workloads.Workload("u1_L24_d5_chi1024", L=24, n_max=4, chi_max=1024, U=HEAD.U, J=HEAD.J,
                                  Jnnn=HEAD.Jnnn, K=HEAD.K, jc=12.5, dt=HEAD.dt, t_end=HEAD.t_end)
        N_HEAD = 12

    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()

    state = head_state(seed=workloads.SEED + rank)
    g = make_head(1, stream.cuda_stream, state)
    for _ in range(args.warmup):
        g.step(1)
        g.measure()
    # the state after the warm-up steps, on the host: the end-to-end loop's input (every arm times
    # the same steps of the evolution, whose cost changes as the synthetic state relaxes)
    torch.cuda.synchronize()
    state_w = ([g.get_site(k)[0] for k in range(HEAD.L)], [g.get_lambda(k) for k in range(HEAD.L + 1)],
               [g.get_charges(k) for k in range(HEAD.L + 1)])
    side = max(1, min(args.steps, SIDE_STEPS))

    # -- device-timed region ------------------------------------------------------
    g.set_option("profile", 1)
    _, l0 = g.counters()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    evs = torch.cuda.Event(enable_timing=True)  # after the first `side` timed steps (the side arms' steps)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            g.step(1)
            g.measure()
            if i + 1 == side:
                evs.record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    ms_side = ev0.elapsed_time(evs)
    _, l1 = g.counters()
    prof = g.profile()
    g.set_option("profile", 0)
    head_bytes = g.device_bytes()
    t_max = max_over_ranks(ms, ws)
    value = job_value(gates_per_step(HEAD.L) * args.steps, ws, t_max / 1e3)

    # -- end to end through the C ABI with host buffers ---------------------------
    # each iteration uploads the post-warm-up state from pinned host memory, takes the first timed
    # step again and reads the observables back
    B, lam, q = state_w
    pinned_B = [torch.from_numpy(np.ascontiguousarray(b)).pin_memory().numpy() for b in B]
    pinned_l = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory().numpy() for x in lam]
    h2d = sum(b.nbytes for b in pinned_B) + sum(x.nbytes for x in pinned_l) + sum(4 * len(x) for x in q)
    d2h = 8 * (HEAD.L + HEAD.L - 1)
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        g.set_state(pinned_B, pinned_l)
        g.set_charges(q)
        g.step(1)
        g.measure()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
    e2e_value = job_value(gates_per_step(HEAD.L) * e2e_steps, ws, e2e_s)
    g.close()

    # -- the plain FP64 and FP64-accurate tensor-core paths on the same state -----------
    fp64 = exact = None
    if not args.no_side:
        side = max(1, min(args.steps, SIDE_STEPS))
        fp64 = side_measurement(time_path, 0, state, stream, side, args.warmup, ws, barrier)
        exact = side_measurement(time_path, 2, state, stream, side, args.warmup, ws, barrier)
        if isinstance(exact, dict) and "error" not in exact:
            exact["note"] = ("precision 2: every large product on the exact-digit tensor-core engine "
                             "(FP64-accurate; parity with the oracle at the FP64 bound)")

    if rank != 0:
        if ws > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # -- roofline of the dominant kernel class ---------------------------------------
    dom = max((k for k in prof if k != "measure"), key=lambda k: prof[k][0])
    dms, dlaunch, dwork = prof[dom]
    achieved = dwork / (dms / 1e3) / 1e12 if dms > 0 and dwork > 0 else None
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops")
    tf32_peak = (bf16 if bf16 else 1900.0) * TF32_RATIO
    if dom in ALU_CLASSES or dom not in ("contract",):
        bound, peak, src = "alu", FP64_PEAK_TFLOPS, \
            "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (FP64 CUDA-core rate; no FP64 entry measured)"
    else:
        bound, peak, src = "tensor", tf32_peak, ("measured bf16_tflops x 1.1/2.25 (nominal tf32/bf16)" if bf16
                                                 else "fallback 1.9 PFLOP/s bf16 x 1.1/2.25")
    traffic, tnote = None, None
    if dom == "tridiag" and args.workload == "L64_d5_chi1024_u1":
        # dram__bytes_read.sum + dram__bytes_write.sum of one k_tridiag_panel launch (the step's first
        # panel, up to 64 charge blocks) from the ncu capture summarised in
        # profiles/k_tridiag_panel_u1_L24_d5_chi1024.md; the same kernel and local sizes as this chain
        traffic = PANEL_LAUNCH_DRAM_BYTES
        tnote = ("DRAM bytes of one k_tridiag_panel launch (first panel of a step, ncu, L=24 chain of the same "
                 "local sizes); the blocks stay L2-resident, the kernel is FP64-pipe and barrier bound")
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic, "traffic_note": tnote,
                "peak_source": src,
                "share_of_step": dms / ms if ms > 0 else None, "launches": dlaunch,
                "work_note": "algorithmic real flops of the class (Hermitian Gram at half, reduction 16/3 b^3 per "
                             "charge block of size b) over its CUDA-event time on the handle's stream"}
    roofline.update(profile_summary(prof))
    if prof["contract"][0] > 0:
        tc_ach = prof["contract"][2] / (prof["contract"][0] / 1e3) / 1e12
        roofline["tensor_kernel"] = {
            "kernel": "k_tf32x3 + FP64 gate product (contract class)", "bound": "tensor", "achieved": tc_ach,
            "peak": tf32_peak, "unit": "TFLOP/s", "frac": tc_ach / tf32_peak, "traffic": None,
            "note": "algorithmic complex flops 8MNK; the 3xTF32 split issues 3x that on the tensor cores"}

    served = None
    if not args.no_served and ws == 1:
        served = side_measurement(served_measurement, stream.cuda_stream)
    batched = None
    if not args.no_batched and ws == 1:
        batched = side_measurement(batched_measurement, stream.cuda_stream)
    dense32 = None
    if not args.no_side and ws == 1:
        dense32 = side_measurement(dense_L32, stream)
    graphm = None
    if not args.no_graph and ws == 1:
        graphm = side_measurement(graph_measurement, stream.cuda_stream)

    cpu = None
    if not args.no_cpu_baseline:
        secs = oracle_update_seconds(state)
        cpu = {"value": 1.0 / secs, "unit": UNIT, "cores": os.cpu_count(), "blas": blas_vendor(), "kind": "oracle",
               "sample": f"one U(1)-oracle gate update of the interior triple on sites 31..33 of the same state "
                         f"(chi_max 1024 on all four bonds), {secs:.1f} s"}

    line = {"metric": METRIC,
            "metric_detail": ("value: mixed path of the particle-number-blocked update (3xTF32 tensor-core "
                              "contractions; decompositions FP64-accurate, their products on the exact-digit "
                              "tensor-core engine); fp64_path: the plain FP64 GPU method on the same state; "
                              "exact_path: FP64-accurate throughout on the tensor cores"),
            "value": value, "unit": UNIT, "svds_per_s": 2.0 * value, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+tf32x3",
            "data": "synthetic", "config": head_config("mixed"),
            "clocks": clk.summary(), "gpu_launches": int(l1 - l0),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps,
                    "note": "every step uploads the post-warm-up state (MPS and bond charges) from pinned host "
                            "memory, takes the first timed step of the evolution again and reads n_j and the "
                            "currents back"},
            "device_bytes": head_bytes,
            "roofline": roofline, "cpu_baseline": cpu, "fp64_path": fp64, "exact_path": exact,
            "mixed_over_fp64": ((fp64["ms_per_step"] / (ms_side / side)) if isinstance(fp64, dict) and
                                fp64.get("ms_per_step") else None),
            "mixed_ms_per_step_side_steps": ms_side / side,
            "dense_L32_d4_chi256": dense32, "served": served, "batched": batched, "graph": graphm}
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
