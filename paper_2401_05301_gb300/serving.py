"""Continuous-batching request loop for TEBD simulations (host-side scheduling).

Requests (a chain, its Hamiltonian parameters, chi_max, dt, number of steps
and measurement interval) arrive over time.  The loop

* admits a waiting request as soon as its device footprint
  (``tebd_estimate_bytes``) fits in the HBM budget and a slot is free,
* keeps every admitted simulation's MPS resident on the GPU,
* advances all admitted simulations together, one second-order step per
  iteration, with ``tebd_batch_step`` (each stage of every layer is one
  grouped launch over the triples of all of them, so newly admitted requests
  share the device with those already running),
* streams n_j and currents back at each request's measurement interval, and
* retires finished simulations, freeing their memory for the next admissions.

Each result is bitwise the same as running the request alone (the batched
kernels treat every triple independently); ``tests/test_gpu_serving.py``
checks this.  Latency = completion time - arrival time.

Failures stay with the requests they hit: a request whose handle cannot be
created or initialised fails alone; a failed batched step fails the requests
in that batch (the library marks every member of a failed batch), whose
handles are closed and whose memory returns to the budget, and serving goes
on.  A request can carry a deadline (latency limit) and can be cancelled with
``Server.cancel``; either ends it at the next step boundary.
"""
from __future__ import annotations

import heapq
import threading
import time
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

from . import binding


@dataclass
class Request:
    rid: int
    arrival: float               # seconds after the loop starts
    L: int
    n_max: int
    chi_max: int
    U: float
    J: float
    Jnnn: float
    K: float
    jc: float
    dt: float
    n_steps: int
    measure_every: int = 10
    occ: Optional[np.ndarray] = None
    w_cut: float = 0.0
    eps_rel: float = 1e-12
    max_slots: int = 0
    deadline_s: Optional[float] = None  # cancelled if not finished this long after arrival
    u1: bool = False                    # the particle-number-blocked form (option "u1")


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float = 0.0
    finished: float = 0.0
    times: list = field(default_factory=list)
    densities: list = field(default_factory=list)
    currents: list = field(default_factory=list)
    gate_updates: int = 0
    status: str = "ok"  # "ok", "failed" or "cancelled"
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class _Active:
    def __init__(self, req: Request, sim: binding.TEBD, nbytes: float, res: Result):
        self.req, self.sim, self.nbytes, self.res = req, sim, nbytes, res
        self.done_steps = 0


class Server:
    """HBM-budgeted continuous batching of TEBD simulations on one GPU."""

    def __init__(self, hbm_budget_bytes: float, precision: int = 1, max_active: int = 64,
                 stream_ptr: Optional[int] = None, on_observables: Optional[Callable] = None,
                 clock: Callable[[], float] = time.perf_counter, sim_factory: Callable = None,
                 step_fn: Callable = None, estimate_fn: Callable = None):
        self.budget = float(hbm_budget_bytes)
        self.precision = int(precision)
        self.max_active = int(max_active)
        self.stream_ptr = stream_ptr
        self.on_observables = on_observables
        self.clock = clock
        self.sim_factory = sim_factory or binding.TEBD
        self.step_fn = step_fn or binding.batch_step
        self.estimate_fn = estimate_fn or binding.estimate_bytes
        self.peak_used = 0.0
        self.peak_active = 0
        self._cancel = set()
        self._lock = threading.Lock()

    def cancel(self, rid: int) -> None:
        """Ask for request rid to end at the next step boundary (safe from other threads
        and from the observables callback); a request not yet admitted never starts."""
        with self._lock:
            self._cancel.add(rid)

    def _cancelled(self, req: Request, now: float) -> str:
        with self._lock:
            if req.rid in self._cancel:
                return "cancelled"
        if req.deadline_s is not None and now - req.arrival > req.deadline_s:
            return "deadline exceeded"
        return ""

    def footprint(self, req: Request) -> float:
        if req.u1:
            return self.estimate_fn(req.L, req.n_max, req.chi_max, req.max_slots, self.precision, u1=True)
        return self.estimate_fn(req.L, req.n_max, req.chi_max, req.max_slots, self.precision)

    def _admit(self, req: Request, now: float) -> _Active:
        kw = {"u1": True} if req.u1 else {}
        sim = self.sim_factory(req.L, req.n_max, req.chi_max, req.U, req.J, req.Jnnn, req.K, req.jc, req.dt,
                               w_cut=req.w_cut, eps_rel=req.eps_rel, precision=self.precision,
                               stream=self.stream_ptr, **kw)
        try:
            if req.max_slots:
                sim.set_option("max_slots", req.max_slots)
            occ = req.occ if req.occ is not None else np.array([1 if j % 2 == 1 else 0 for j in range(1, req.L + 1)])
            sim.init_product(occ)
        except Exception:
            sim.close()
            raise
        return _Active(req, sim, self.footprint(req), Result(req.rid, req.arrival, admitted=now))

    def run(self, requests) -> dict:
        """Serve every request; returns {rid: Result} once all have finished, failed or
        been cancelled (Result.status)."""
        pending = [(r.arrival, r.rid, r) for r in requests]
        heapq.heapify(pending)
        for r in requests:
            if self.footprint(r) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the whole HBM budget")
        active: list[_Active] = []
        results: dict[int, Result] = {}
        used = 0.0
        t0 = self.clock()

        def end(a: _Active, status: str, error: str, now: float):
            nonlocal used
            a.res.status, a.res.error, a.res.finished = status, error, now
            results[a.req.rid] = a.res
            a.sim.close()
            used -= a.nbytes

        while pending or active:
            now = self.clock() - t0
            # cancellations and deadlines, at a step boundary
            if any(self._cancelled(p[2], now) for p in pending):
                keep = []
                for p in pending:
                    why = self._cancelled(p[2], now)
                    if why:
                        results[p[1]] = Result(p[1], p[0], admitted=now, finished=now, status="cancelled", error=why)
                    else:
                        keep.append(p)
                pending = keep
                heapq.heapify(pending)
            still = []
            for a in active:
                why = self._cancelled(a.req, now)
                if why:
                    end(a, "cancelled", why, now)
                else:
                    still.append(a)
            active = still
            if not active:
                used = 0.0  # no rounding residue may keep a request that fits the budget waiting
            # admit in arrival order while the budget and the slot count allow
            while pending and pending[0][0] <= now and len(active) < self.max_active:
                req = pending[0][2]
                need = self.footprint(req)
                if used + need > self.budget:
                    break
                heapq.heappop(pending)
                try:
                    act = self._admit(req, now)
                except Exception as e:  # this request alone fails; its memory was never counted
                    results[req.rid] = Result(req.rid, req.arrival, admitted=now, finished=now, status="failed",
                                              error=str(e))
                    continue
                active.append(act)
                used += need
                self.peak_used = max(self.peak_used, used)
                self.peak_active = max(self.peak_active, len(active))
            if not active:
                if pending:  # idle until the next arrival
                    time.sleep(max(0.0, min(0.01, pending[0][0] - now)))
                continue
            try:
                # one batched step per form (the library batches simulations of one form together)
                groups = {}
                for a in active:
                    groups.setdefault(a.req.u1, []).append(a.sim)
                for sims in groups.values():
                    self.step_fn(sims, 1)
            except Exception as e:  # the library fails every member of a failed batch
                now = self.clock() - t0
                for a in active:
                    end(a, "failed", str(e), now)
                active = []
                continue
            now = self.clock() - t0
            still = []
            for a in active:
                a.done_steps += 1
                if a.done_steps % a.req.measure_every == 0 or a.done_steps == a.req.n_steps:
                    try:
                        n, cur = a.sim.measure()
                    except Exception as e:
                        end(a, "failed", str(e), self.clock() - t0)
                        continue
                    a.res.times.append(a.done_steps * a.req.dt)
                    a.res.densities.append(n)
                    a.res.currents.append(cur)
                    if self.on_observables:
                        self.on_observables(a.req.rid, a.done_steps * a.req.dt, n, cur)
                if a.done_steps >= a.req.n_steps:
                    a.res.gate_updates = a.sim.counters()[0]
                    end(a, "ok", "", self.clock() - t0)
                else:
                    still.append(a)
            active = still
        with self._lock:  # cancellations belong to this run's requests
            self._cancel.clear()
        return results


def run_alone(req: Request, precision: int = 1, stream_ptr: Optional[int] = None) -> Result:
    """The same request on its own handle, stepped alone (reference for the mix)."""
    srv = Server(float("inf"), precision=precision, stream_ptr=stream_ptr)
    r = Request(**{**req.__dict__, "arrival": 0.0})
    return srv.run([r])[req.rid]


def latency_stats(results: dict) -> dict:
    """p50/p99/mean latency and throughput over the requests that finished; counts of the
    failed and cancelled ones beside them."""
    ok = [r for r in results.values() if r.status == "ok"]
    out = {"failed": sum(r.status == "failed" for r in results.values()),
           "cancelled": sum(r.status == "cancelled" for r in results.values())}
    if not ok:
        return {"p50_s": None, "p99_s": None, "mean_s": None, "requests": 0, "gate_updates": 0,
                "throughput_gate_updates_per_s": None, "span_s": 0.0, **out}
    lat = np.array([r.latency for r in ok])
    gates = sum(r.gate_updates for r in ok)
    span = max(r.finished for r in ok) - min(r.arrival for r in ok)
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "requests": len(lat), "gate_updates": int(gates),
            "throughput_gate_updates_per_s": gates / span if span > 0 else None, "span_s": span, **out}


def poisson_requests(n: int, rate_per_s: float, seed: int, make: Callable[[int, float, np.random.Generator], Request]):
    """n requests with exponential inter-arrival times (seeded); make(i, t, rng) builds each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += float(rng.exponential(1.0 / rate_per_s))
        out.append(make(i, t, rng))
    return out
