"""Host logic of the serving loop (admission by HBM budget, continuous batching,
retirement, latency statistics) with a fake simulation: no GPU."""
import numpy as np
import pytest

from paper_2401_05301_gb300 import serving


class FakeSim:
    def __init__(self, L, n_max, chi_max, U, J, Jnnn, K, jc, dt, **kw):
        self.L, self.steps, self.closed = L, 0, False

    def set_option(self, k, v):
        pass

    def init_product(self, occ):
        self.occ = np.asarray(occ, dtype=float)

    def measure(self):
        return self.occ + self.steps, np.zeros(self.L - 1)

    def counters(self):
        return 10 * self.steps, 0

    def close(self):
        self.closed = True


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


def _server(budget, clock, log):
    def step(sims, n):
        log.append(len(sims))
        for s in sims:
            s.steps += n
        clock.t += 0.1
    return serving.Server(budget, sim_factory=FakeSim, step_fn=step, clock=clock,
                          estimate_fn=lambda L, n_max, chi, slots, precision: 1.0 * L)


def _req(i, t, L, steps):
    return serving.Request(rid=i, arrival=t, L=L, n_max=2, chi_max=8, U=1, J=1, Jnnn=0, K=0, jc=1, dt=0.1,
                           n_steps=steps, measure_every=2)


def test_budget_and_continuous_admission():
    clock, log = FakeClock(), []
    srv = _server(20.0, clock, log)
    reqs = [_req(0, 0.0, 8, 4), _req(1, 0.0, 8, 6), _req(2, 0.05, 8, 2), _req(3, 0.3, 4, 2)]
    res = srv.run(reqs)
    assert sorted(res) == [0, 1, 2, 3]
    assert srv.peak_used <= 20.0
    assert log[0] == 2  # the third request waited for memory
    assert max(log) == 3  # ... then joined request 1's running batch together with request 3
    assert res[2].admitted >= res[0].finished  # admitted when request 0 retired
    # continuous batching: request 3 joined while request 1 was still running
    assert res[3].admitted < res[1].finished
    for r in res.values():
        assert r.finished >= r.arrival and len(r.densities) >= 1
    st = serving.latency_stats(res)
    assert st["requests"] == 4 and st["p99_s"] >= st["p50_s"] > 0


def test_oversized_request_is_rejected():
    clock, log = FakeClock(), []
    srv = _server(5.0, clock, log)
    try:
        srv.run([_req(0, 0.0, 8, 2)])
    except ValueError:
        return
    raise AssertionError("expected a ValueError")


def test_poisson_stream_is_seeded():
    mk = lambda i, t, rng: _req(i, t, 8, 2)
    a = serving.poisson_requests(5, 10.0, 7, mk)
    b = serving.poisson_requests(5, 10.0, 7, mk)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))


# -- failures, deadlines and cancellation stay with their requests ------------------

def _tracking_server(budget, clock, log, created, fail_create=(), fail_init=(), fail_step_at=None,
                     fail_measure=()):
    class Sim(FakeSim):
        def __init__(self, L, *a, **kw):
            rid = len(created)
            if rid in fail_create:
                created.append(None)
                raise RuntimeError("tebd_create: out of device memory (status -2)")
            super().__init__(L, *a, **kw)
            self.rid = rid
            created.append(self)

        def init_product(self, occ):
            if self.rid in fail_init:
                raise RuntimeError("tebd_init_product: invalid argument (status -1)")
            super().init_product(occ)

        def measure(self):
            if self.rid in fail_measure:
                raise RuntimeError("tebd_measure: non-finite singular values (status -7)")
            return super().measure()

    calls = [0]

    def step(sims, n):
        calls[0] += 1
        log.append(sorted(s.rid for s in sims))
        clock.t += 0.1
        if fail_step_at is not None and calls[0] == fail_step_at:
            raise RuntimeError("tebd_batch_step: non-finite singular values (status -7)")
        for s in sims:
            s.steps += n

    return serving.Server(budget, sim_factory=Sim, step_fn=step, clock=clock,
                          estimate_fn=lambda L, n_max, chi, slots, precision: 1.0 * L)


def test_failed_admission_fails_that_request_only():
    """Handle creation refused (request 1) and initialisation refused (request 2): those two fail,
    their handles are closed, no budget is held for them, and the rest are served."""
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(16.0, clock, log, created, fail_create={1}, fail_init={2})
    res = srv.run([_req(i, 0.0, 8, 2) for i in range(4)])
    assert {r: res[r].status for r in res} == {0: "ok", 1: "failed", 2: "failed", 3: "ok"}
    assert "status -2" in res[1].error and "status -1" in res[2].error
    assert created[2].closed and created[1] is None
    assert srv.peak_used <= 16.0
    assert log[0] == [0, 3]  # requests 0 and 3 ran together: the failed ones held no memory
    st = serving.latency_stats(res)
    assert st["requests"] == 2 and st["failed"] == 2 and st["cancelled"] == 0


def test_failed_batch_fails_its_members_and_serving_continues():
    """The second batched step fails: the two requests in it fail and are closed; a request
    waiting for memory is then admitted into the freed budget and finishes."""
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(16.0, clock, log, created, fail_step_at=2)
    res = srv.run([_req(0, 0.0, 8, 4), _req(1, 0.0, 8, 4), _req(2, 0.05, 8, 2)])
    assert res[0].status == res[1].status == "failed" and "status -7" in res[0].error
    assert created[0].closed and created[1].closed
    assert res[2].status == "ok" and res[2].admitted >= res[0].finished
    assert log == [[0, 1], [0, 1], [2], [2]]


def test_failed_measurement_fails_that_request_only():
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(16.0, clock, log, created, fail_measure={0})
    res = srv.run([_req(0, 0.0, 8, 4), _req(1, 0.0, 8, 4)])
    assert res[0].status == "failed" and res[1].status == "ok"
    assert len(res[1].densities) == 2 and created[0].closed
    assert log == [[0, 1], [0, 1], [1], [1]]  # request 0 left after its first measurement


def test_deadline_cancels_a_slow_request_and_frees_its_memory():
    """Request 0 needs 10 steps (1 s of fake time) but has a 0.35 s deadline: it is cancelled at
    the step boundary after the deadline, and request 1, waiting for memory, then runs."""
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(8.0, clock, log, created)
    r0 = _req(0, 0.0, 8, 10)
    r0.deadline_s = 0.35
    res = srv.run([r0, _req(1, 0.0, 8, 2)])
    assert res[0].status == "cancelled" and res[0].error == "deadline exceeded"
    assert created[0].closed and created[0].steps == 4
    assert res[1].status == "ok" and res[1].admitted >= res[0].finished
    assert serving.latency_stats(res)["cancelled"] == 1


def test_cancel_before_admission_and_while_running():
    """cancel() of a request not yet admitted: it never starts.  cancel() from the observables
    callback: the request ends at the next step boundary; the other one is unaffected."""
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(16.0, clock, log, created)
    srv.cancel(2)
    srv.on_observables = lambda rid, t, n, cur: srv.cancel(0) if rid == 0 else None
    res = srv.run([_req(0, 0.0, 8, 8), _req(1, 0.0, 8, 4), _req(2, 0.0, 8, 2)])
    assert res[2].status == "cancelled" and all(s is None or s.rid != 2 for s in created)
    assert res[0].status == "cancelled" and created[0].steps == 2 and created[0].closed
    assert res[1].status == "ok" and len(res[1].densities) == 2
    assert log == [[0, 1], [0, 1], [1], [1]]


@pytest.mark.timeout(30)
def test_budget_rounding_cannot_stall_admission():
    """Footprints 0.1 and 0.2 run together and retire, leaving 0.1 + 0.2 - 0.1 - 0.2 = 2.8e-17
    in the running sum; a request of exactly the whole budget (0.31) must still be admitted
    once nothing runs (without the reset it would wait forever)."""
    clock, log = FakeClock(), []
    sizes = {8: 0.1, 4: 0.2, 2: 0.31}

    def step(sims, n):
        log.append(len(sims))
        for s in sims:
            s.steps += n
        clock.t += 0.1
    srv = serving.Server(0.31, sim_factory=FakeSim, step_fn=step, clock=clock,
                         estimate_fn=lambda L, n_max, chi, slots, precision: sizes[L])
    res = srv.run([_req(0, 0.0, 8, 2), _req(1, 0.0, 4, 2), _req(2, 0.0, 2, 2)])
    assert all(r.status == "ok" for r in res.values()) and log == [2, 2, 1, 1]


def test_cancellations_do_not_outlive_their_run():
    clock, log, created = FakeClock(), [], []
    srv = _tracking_server(16.0, clock, log, created)
    srv.cancel(0)
    assert srv.run([_req(0, 0.0, 8, 2)])[0].status == "cancelled"
    assert srv.run([_req(0, 0.0, 8, 2)])[0].status == "ok"  # the same id in a later run is served
