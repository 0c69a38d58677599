"""Plant plausible mistakes in the oracle and check that a pin catches each one.

Each mutation is a small change a reader could make by accident (a wrong sign,
a dropped factor, a transposed operand, a wrong bond index, a non-symmetric
layer order).  The pins of ``test_oracle_pins`` are re-run in miniature on the
mutated oracle and must fail.
"""
import numpy as np
import pytest

from oracle import ed, model
from oracle import tebd as tebd_mod
from oracle.tebd import TEBD
import workloads


def _split_error(three_site_term, L=5, n_max=2):
    U, J, Jnnn, K, jc = 2.0, 1.0, 0.3, 0.1, 3.3
    basis, index = ed.full_basis(L, n_max)
    H = ed.hamiltonian(basis, index, L, n_max, U, J, Jnnn, K, jc)
    S = sum(ed.embed_three_site(three_site_term(j, L, n_max, U, J, Jnnn, K, jc), j - 1, L, n_max + 1)
            for j in range(1, L - 1))
    return np.max(np.abs(S - H))


def _dense_error(cls=TEBD, schedule=model.step_schedule, L=6, n_max=2, steps=6):
    dt = 0.05
    T = cls(L, n_max, 10 ** 6, 3.0, 1.0, 0.2, 0.05, 3.2, dt, w_cut=0.0, eps_rel=1e-24)
    occ = workloads.cdw(L)
    T.init_product(occ)
    psi = ed.dense_product(occ, n_max + 1)
    for _ in range(steps):
        T.step()
        psi = ed.dense_trotter_step(psi, T.gate, model.step_schedule(L, dt), n_max + 1)
    n_d, C_d = ed.dense_observables(psi)
    return max(np.max(np.abs(T.densities() - n_d)), np.max(np.abs(T.correlators() - C_d)))


def test_reference_is_clean():
    assert _split_error(model.three_site_term) < 1e-13
    assert _dense_error() < 1e-12


def test_catches_nnn_sign_flip():
    def bad(j, L, n_max, U, J, Jnnn, K, jc):
        return model.three_site_term(j, L, n_max, U, J, -Jnnn, K, jc)
    assert _split_error(bad) > 1e-3


def test_catches_dropped_bond_sharing():
    orig = model.bond_multiplicity
    try:
        model.bond_multiplicity = lambda k, L: 1
        assert _split_error(model.three_site_term) > 1e-3
    finally:
        model.bond_multiplicity = orig


def test_catches_adjoint_gate():
    """G^+ instead of G (h is real symmetric, so G.T == G and only the adjoint shows)."""
    class Bad(TEBD):
        def apply_gate(self, i, G):
            return super().apply_gate(i, G.conj().T)
    assert _dense_error(Bad) > 1e-4


def test_catches_wrong_lambda_in_densities():
    class Bad(TEBD):
        def densities(self):
            out = np.empty(self.L)
            sv = np.arange(self.d, dtype=np.float64)
            for k in range(self.L):
                w = (self.lam[k + 1] ** 2)[None, None, :] * np.abs(self.B[k]) ** 2
                out[k] = np.sum(w.sum(axis=(0, 2)) * sv)
            return out
    assert _dense_error(Bad) > 1e-4


def test_catches_missing_renormalisation():
    class Bad(TEBD):
        def _truncated_svd(self, M):
            U, s, Vh = tebd_mod.svd_desc(M)
            k, w = tebd_mod.truncation_rule(s, self.chi_max, self.w_cut, self.eps_rel)
            return s[:k], Vh[:k], 1.0, w
    T = Bad(8, 3, 6, 5.0, 1.0, 0.12, 0.005, 4.5, 0.01, w_cut=1e-10, eps_rel=1e-12)
    T.init_product(workloads.cdw(8))
    T.step(100)
    assert max(abs(np.sum(l ** 2) - 1.0) for l in T.lam) > 1e-8


def test_catches_first_order_schedule():
    """A-B-C (first order) instead of A/2 B/2 C B/2 A/2: the dt-halving ratio drops to ~2."""
    def first_order(L, dt):
        trip = {lab: [j for j in range(1, L - 1) if model.layer_of(j) == lab] for lab in "ABC"}
        return [(trip["A"], dt), (trip["B"], dt), (trip["C"], dt)]
    wl = workloads.PARITY_L8
    occ = wl.occupation()
    ex = ed.SectorED(wl.L, wl.n_max, occ, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    n_ex, _ = ex.observables(0.5)
    orig = model.step_schedule
    errs = []
    try:
        model.step_schedule = first_order
        for dt in (0.05, 0.025):
            T = TEBD(wl.L, wl.n_max, 256, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, dt, eps_rel=1e-24)
            T.init_product(occ)
            T.step(int(round(0.5 / dt)))
            errs.append(np.max(np.abs(T.densities() - n_ex)))
    finally:
        model.step_schedule = orig
    assert not (3.5 <= errs[0] / errs[1] <= 4.5)



def test_catches_wrong_fourth_order_weights():
    """Middle weight 1 - 2p instead of 1 - 4p: the 4th-order step no longer spans dt,
    and the exact-ED comparison of the convergence pin fails by orders of magnitude."""
    good = model.step_schedule

    def bad(L, dt, order=2):
        if order != 4:
            return good(L, dt, order)
        p = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
        return good(L, p * dt) * 2 + good(L, (1.0 - 2.0 * p) * dt) + good(L, p * dt) * 2

    wl = workloads.PARITY_L8
    occ = wl.occupation()
    ex = ed.SectorED(wl.L, wl.n_max, occ, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    n_ex, _ = ex.observables(1.0)
    T = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, 0.05, eps_rel=1e-24, order=4)
    try:
        model.step_schedule = bad
        T.init_product(occ)
        T.step(20)
    finally:
        model.step_schedule = good
    assert np.max(np.abs(T.densities() - n_ex)) > 1e-3  # the correct split is within 2.3e-7 here


def _two_boson_error(three_site_term, U=2.5, J=0.9):
    """Distance of the closed-form two-boson levels (U +- sqrt(U^2 + 8 J^2))/2 from the
    spectrum of the L = 3 term (the closed-form pin, in miniature)."""
    ev = np.linalg.eigvalsh(three_site_term(1, 3, 2, U, J, 0.0, 0.0, 2.0))
    r = np.sqrt(U * U + 8 * J * J)
    return max(np.min(np.abs(ev - x)) for x in ((U + r) / 2, (U - r) / 2))


def test_catches_doubled_interaction_read_into_both_builders():
    """U n(n-1) instead of U/2 n(n-1), misread into eq. (1) itself: the Fock-basis split
    pin cannot see a mistake both builders share; the closed-form spectrum does."""
    def bad(j, L, n_max, U, J, Jnnn, K, jc):
        return model.three_site_term(j, L, n_max, 2 * U, J, Jnnn, K, jc)
    assert _two_boson_error(model.three_site_term) < 1e-12
    assert _two_boson_error(bad) > 1e-2


def test_catches_missing_sqrt_n_in_annihilator():
    orig = model.local_ops

    def bad_ops(n_max):
        b, num, one = orig(n_max)
        return (b != 0).astype(b.dtype), num, one
    try:
        model.local_ops = bad_ops
        assert _two_boson_error(model.three_site_term) > 1e-2
    finally:
        model.local_ops = orig


def test_catches_dropped_interaction():
    """The on-site U term left out: the d = 3 chain is then (up to the n_max cap) free bosons,
    whose densities from singly occupied sites equal the free-fermion ones, so the deviation
    no longer falls by 4 per doubling of U."""
    from oracle import free
    orig = model.three_site_term

    def bad(j, L, n_max, U, J, Jnnn, K, jc):
        return orig(j, L, n_max, 0.0, J, Jnnn, K, jc)
    L, occ = 8, workloads.cdw(8)
    n_free, _ = free.observables(free.propagator(free.one_body_h(L, 1.0, 0.0, 0.0, 4.5), 0.5), occ)
    devs = []
    try:
        model.three_site_term = bad
        for U in (20.0, 40.0):
            T = TEBD(L, 2, 256, U, 1.0, 0.0, 0.0, 4.5, 0.01, eps_rel=1e-14)
            T.init_product(occ)
            T.step(50)
            devs.append(np.max(np.abs(T.densities() - n_free)))
    finally:
        model.three_site_term = orig
    assert not (3.6 < devs[0] / devs[1] < 4.4), devs
