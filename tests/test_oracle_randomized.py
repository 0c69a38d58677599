"""Pins of the randomized-range-finder truncation (the cheaper SVD of Sec. V).

Checked against exact SVDs (exactly low-rank input), against what the range
finder's analysis fixes (power iterations push the range error down to the
optimal sigma_{l+1}), against reading T on full spectra, and against the dense
oracle in TEBD runs with and without a chi_max cut.
"""
import numpy as np
import pytest

import workloads
from oracle.randomized import RandomizedTEBD, randomized_svd, truncation_rule_partial
from oracle.tebd import TEBD, truncation_rule


def _omega(n, l, call):
    return workloads.gaussian_test_matrix(n, l, call)


def test_exact_for_exactly_low_rank_input():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((300, 25)) + 1j * rng.standard_normal((300, 25))
    B = rng.standard_normal((25, 500)) + 1j * rng.standard_normal((25, 500))
    M = A @ B
    U, s, Vh = randomized_svd(M, _omega(500, 35, 0), q=0)
    s_ex = np.linalg.svd(M, compute_uv=False)
    assert np.max(np.abs(s[:25] - s_ex[:25])) < 1e-13 * s_ex[0]
    assert np.linalg.norm(M - U @ (U.conj().T @ M)) < 1e-13 * np.linalg.norm(M)
    assert np.max(np.abs((U[:, :25] * s[:25]) @ Vh[:25] - M)) < 1e-12 * s_ex[0]


def test_power_iterations_reach_the_optimal_range():
    """Geometric spectrum sigma_i = 2^(-i/4): with a sketch of l = 30 the range error can be no
    smaller than sigma_31; two power iterations bring it within a factor 2 of that, and the leading
    20 singular values converge as the iterations grow (~2e-2, ~2e-5, ~2e-8 relative)."""
    rng = np.random.default_rng(2)
    m, n, l = 200, 400, 30
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, m)))
    sig = 2.0 ** (-np.arange(m) / 4)
    M = (Q1 * sig) @ Q2.T
    top = []
    for q in (0, 1, 2):
        U, s, _ = randomized_svd(M, _omega(n, l, 1), q=q)
        err = np.linalg.norm(M - U @ (U.conj().T @ M), 2)
        assert err >= sig[l] * (1 - 1e-12)  # no rank-l range does better (Eckart-Young)
        top.append(np.max(np.abs(s[:20] - sig[:20]) / sig[:20]))
        if q == 2:
            assert err <= 2.0 * sig[l]
    assert top[0] > top[1] > top[2] and top[2] < 1e-6


@pytest.mark.parametrize("case", [
    (np.sqrt(np.array([0.5, 0.3, 0.2 - 1e-11, 1e-11])), 10, 1e-10, 1e-14),
    (np.sqrt(np.array([0.5, 0.3, 0.2 - 1e-11, 1e-11])), 2, 0.0, 1e-14),
    (np.sqrt(np.array([0.5, 0.3, 0.2 - 1e-11, 1e-11])), 10, 0.0, 2e-11),
    (np.array([1.0, 0.0, 0.0]), 10, 0.0, 1e-12),
    (np.exp(-np.arange(40) / 3.0), 25, 1e-8, 1e-12),
])
def test_partial_rule_equals_reading_t_on_full_spectra(case):
    s, chi_max, w_cut, eps = case
    k, w = truncation_rule_partial(s, float(np.sum(s ** 2)), chi_max, w_cut, eps)
    k0, w0 = truncation_rule(s, chi_max, w_cut, eps)
    assert k == k0 and abs(w - w0) < 1e-15


def test_full_sketch_is_an_exact_svd():
    """l = min(m, n): the sampled range is the whole range, so the singular values equal LAPACK's
    to rounding (1e-13 of sigma_1) and the triplets rebuild M, even with tiny singular values."""
    rng = np.random.default_rng(3)
    m, n = 64, 256
    Q1, _ = np.linalg.qr(rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m)))
    sig = 10.0 ** (-np.linspace(0, 14, m))
    M = (Q1 * sig) @ Q2.conj().T
    for q in (0, 2):
        U, s, Vh = randomized_svd(M, _omega(n, m, 5), q=q)
        assert np.max(np.abs(s - sig)) < 1e-13
        assert np.max(np.abs((U * s) @ Vh - M)) < 1e-13


def test_untruncated_run_matches_the_dense_oracle():
    """chi_max = 256 above every rank at the paper's eps = 1e-12: the same chi' and observables
    as exact SVDs within 1e-12 over t = 1.  (With eps = 1e-24 the runs keep singular values at
    rounding level, whose vectors any second decomposition route moves; those components then
    grow like sqrt(p), the mechanism of reading F, so both routes part at ~1e-10.)"""
    wl = workloads.PARITY_L8
    args = (wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt)
    r = RandomizedTEBD(*args, w_cut=0.0, eps_rel=1e-12, omega_fn=_omega)
    o = TEBD(*args, w_cut=0.0, eps_rel=1e-12)
    r.init_product(wl.occupation())
    o.init_product(wl.occupation())
    r.step(100)
    o.step(100)
    assert r.chi() == o.chi()
    assert np.max(np.abs(r.densities() - o.densities())) < 1e-12
    assert np.max(np.abs(r.currents() - o.currents())) < 1e-12


def test_truncating_run_keeps_the_dense_decisions():
    """chi_max = 16 on L = 8 for t = 1: the same chi' everywhere as exact SVDs, observables within
    1e-12, and the discarded weight within 1e-3 relative (its tail comes from the sketched values)."""
    wl = workloads.PARITY_L8
    args = (wl.L, wl.n_max, 16, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt)
    r = RandomizedTEBD(*args, w_cut=0.0, eps_rel=1e-12, omega_fn=_omega)
    o = TEBD(*args, w_cut=0.0, eps_rel=1e-12)
    r.init_product(wl.occupation())
    o.init_product(wl.occupation())
    r.step(100)
    o.step(100)
    assert r.chi() == o.chi() and o.w_total > 1e-10
    assert np.max(np.abs(r.densities() - o.densities())) < 1e-12
    assert np.max(np.abs(r.currents() - o.currents())) < 1e-12
    assert abs(r.w_total - o.w_total) < 1e-3 * o.w_total


def test_test_matrices_are_an_input():
    with pytest.raises(ValueError):
        RandomizedTEBD(6, 2, 16, 1.0, 1.0, 0.1, 0.0, 3.5, 0.01)
    a, b = _omega(10, 4, 3), _omega(10, 4, 3)
    assert np.array_equal(a, b) and not np.array_equal(a, _omega(10, 4, 4))


def test_mutation_tail_from_the_sketch_is_caught(monkeypatch):
    """A planted mistake: rule T's total taken from the sketched values (sum of s^2 over the l
    computed values) instead of ||theta'||_F^2.  With a sketch of exactly chi_max = 16 columns the
    discarded weight then reads zero, far outside the 1e-3 of the dense oracle's that the pin above
    allows (the correct total gives the exact tail for any sketch size)."""
    from oracle import randomized as rmod

    def bad(self, M):
        m, n = M.shape
        l = min(self.chi_max + self.oversample, m, n)
        omega = self.omega_fn(n, l, self.calls)
        self.calls += 1
        _, s, Vh = rmod.randomized_svd(M, omega, self.power_iters)
        total = float(np.sum(s * s))
        k, w = rmod.truncation_rule_partial(s, total, self.chi_max, self.w_cut, self.eps_rel)
        s = s[:k]
        norm = np.sqrt(np.sum(s * s))
        return s / norm, Vh[:k], norm, w

    monkeypatch.setattr(RandomizedTEBD, "_truncated_svd", bad)
    wl = workloads.PARITY_L8
    args = (wl.L, wl.n_max, 16, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt)
    r = RandomizedTEBD(*args, w_cut=0.0, eps_rel=1e-12, omega_fn=_omega, oversample=0, power_iters=2)
    o = TEBD(*args, w_cut=0.0, eps_rel=1e-12)
    r.init_product(wl.occupation())
    o.init_product(wl.occupation())
    r.step(100)
    o.step(100)
    assert abs(r.w_total - o.w_total) > 1e-3 * o.w_total
