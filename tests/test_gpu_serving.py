"""Batched and served forms on the GPU.

* tebd_batch_step over uneven simulations (different L, d, chi_max,
  parameters) gives bitwise the same observables as stepping each alone.
* The continuous-batching server: every request's streamed observables are
  the same in the mix as alone (tolerance 1e-12, expected exact), admission
  keeps the HBM budget, and latency statistics are produced.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIMS = [  # L, n_max, chi_max, U, J, Jnnn, K, jc, dt, w_cut
    (9, 2, 32, 2.0, 1.0, 0.1, 0.01, 5.0, 0.02, 1e-10),
    (12, 3, 64, 5.0, 1.0, 0.12, 0.005, 6.5, 0.01, 0.0),
    (16, 1, 16, 7.0, 1.0, 0.0, 0.002, 8.5, 0.02, 1e-9),
    (7, 4, 128, 3.0, 1.0, 0.05, 0.0, 4.0, 0.01, 0.0),
]


def _make(p, precision):
    from paper_2401_05301_gb300 import TEBD
    L, n_max, chi, U, J, Jnnn, K, jc, dt, wc = p
    g = TEBD(L, n_max, chi, U, J, Jnnn, K, jc, dt, w_cut=wc, precision=precision)
    g.init_product([1 if j % 2 == 1 else 0 for j in range(1, L + 1)])
    return g


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_is_bitwise_the_same_as_alone(lib, precision):
    from paper_2401_05301_gb300 import batch_step
    alone = []
    for p in SIMS:
        g = _make(p, precision)
        g.step(15)
        alone.append(np.concatenate(g.measure()))
        g.close()
    sims = [_make(p, precision) for p in SIMS]
    for _ in range(3):
        batch_step(sims, 5)
    for g, ref, p in zip(sims, alone, SIMS):
        got = np.concatenate(g.measure())
        assert np.array_equal(got, ref)
        assert abs(g.stats()[0] - 15 * p[8]) < 1e-12
        g.close()


def test_server_mix_matches_alone(lib):
    from paper_2401_05301_gb300 import serving

    def make(i, t, rng):
        L = int(rng.choice([8, 10, 12]))
        return serving.Request(rid=i, arrival=t, L=L, n_max=int(rng.choice([2, 3])), chi_max=int(rng.choice([16, 32])),
                               U=float(rng.uniform(2, 6)), J=1.0, Jnnn=float(rng.uniform(0, 0.15)),
                               K=float(rng.uniform(0, 0.01)), jc=(L + 1) / 2, dt=0.01,
                               n_steps=int(rng.integers(10, 30)), measure_every=5, w_cut=1e-10)

    reqs = serving.poisson_requests(6, 40.0, 240105301, make)
    budget = 2.2 * max(serving.Server(1).footprint(r) for r in reqs)
    srv = serving.Server(budget, precision=1)
    mixed = srv.run(reqs)
    assert sorted(mixed) == [r.rid for r in reqs]
    assert srv.peak_used <= budget
    assert srv.peak_active >= 2  # requests really shared the device
    for r in reqs:
        alone = serving.run_alone(r, precision=1)
        m = mixed[r.rid]
        assert len(m.densities) == len(alone.densities)
        for a, b in zip(m.densities + m.currents, alone.densities + alone.currents):
            assert np.max(np.abs(a - b)) <= 1e-12
    st = serving.latency_stats(mixed)
    print("served:", st)
    assert st["p99_s"] >= st["p50_s"] > 0
