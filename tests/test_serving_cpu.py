"""Host logic of the serving loop (admission by HBM budget, continuous batching,
retirement, latency statistics) with a fake simulation: no GPU."""
import numpy as np

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
