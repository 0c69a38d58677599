"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: eq. (1)
assembled independently in the Fock basis, exact diagonalisation, library
routines (expm), free-particle closed forms and conservation laws.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import ed, free, model
from oracle.tebd import TEBD, truncation_rule
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _tebd(wl, **kw):
    args = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K,
                jc=wl.jc, dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    args.update(kw)
    return TEBD(**args)


# -- eq. (1) and its three-site split ---------------------------------------------

@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_three_site_split_sums_to_eq1(L):
    """sum_j h_j (reading S) equals eq. (1) built directly in the Fock basis."""
    rng = np.random.default_rng(L)
    n_max = 2
    d = n_max + 1
    U, J, Jnnn, K = rng.uniform(0.5, 3, size=4)
    jc = (L + 1) / 2 + 0.3
    basis, index = ed.full_basis(L, n_max)
    H = ed.hamiltonian(basis, index, L, n_max, U, J, Jnnn, K, jc)
    S = sum(ed.embed_three_site(model.three_site_term(j, L, n_max, U, J, Jnnn, K, jc), j - 1, L, d)
            for j in range(1, L - 1))
    assert np.max(np.abs(S - H)) < 1e-13


def test_gate_is_exact_exponential():
    """G = exp(-i h tau): compare with scipy expm and check unitarity."""
    h = model.three_site_term(2, 6, 3, 5.0, 1.0, 0.1, 0.01, 3.5)
    for tau in (0.005, 0.01, 0.3):
        G = model.gate(h, tau)
        assert np.max(np.abs(G - scipy.linalg.expm(-1j * tau * h))) < 1e-13
        assert np.max(np.abs(G.conj().T @ G - np.eye(len(G)))) < 1e-13


def test_sector_dimension_reading_E():
    """N = 4 bosons on L = 8: C(11,4) = 330 states without a cap, 322 with n_max = 3."""
    assert len(ed.sector_basis(8, 4, 4)[0]) == 330
    assert len(ed.sector_basis(8, 3, 4)[0]) == 322


def test_schedule_covers_each_triple_with_total_time_dt():
    """Layers A/2 B/2 C B/2 A/2: every triple gets total time dt; layers are disjoint."""
    L, dt = 11, 0.01
    tot = {}
    for triples, tau in model.step_schedule(L, dt):
        sites = [s for j in triples for s in (j, j + 1, j + 2)]
        assert len(sites) == len(set(sites))
        for j in triples:
            tot[j] = tot.get(j, 0.0) + tau
    assert sorted(tot) == list(range(1, L - 1))
    assert all(abs(v - dt) < 1e-15 for v in tot.values())


# -- truncation rule (reading T) ------------------------------------------------------

def test_truncation_rule_cases():
    s = np.sqrt(np.array([0.5, 0.3, 0.2 - 1e-11, 1e-11]))
    assert truncation_rule(s, 10, 1e-10, 1e-14)[0] == 3
    chi, w = truncation_rule(s, 10, 1e-10, 1e-14)
    assert abs(w - 1e-11) < 1e-20
    assert truncation_rule(s, 2, 0.0, 1e-14) == (2, pytest.approx(0.2))
    assert truncation_rule(s, 10, 0.0, 1e-12)[0] == 4
    assert truncation_rule(s, 10, 0.0, 2e-11)[0] == 3  # eps floor drops p = 1e-11
    assert truncation_rule(np.array([1.0, 0.0, 0.0]), 10, 0.0, 1e-12)[0] == 1
    # unnormalised input: rule works on p = s^2 / sum s^2
    assert truncation_rule(3.0 * s, 10, 1e-10, 1e-14)[0] == 3


# -- MPS machinery vs dense Trotterised evolution ----------------------------------

def _dense_run(wl, occ, n_steps, tebd):
    d = wl.d
    psi = ed.dense_product(occ, d)
    sched = model.step_schedule(wl.L, wl.dt)
    for _ in range(n_steps):
        psi = ed.dense_trotter_step(psi, tebd.gate, sched, d)
    return psi


def test_tebd_matches_dense_trotter_L8():
    """L=8, d=4, chi_max=256 (no truncation): TEBD == dense Trotterised state to 1e-12.

    The floor eps_rel = 1e-24 keeps every singular value above LAPACK's noise:
    with the paper's eps = 1e-12 floor the run drifts from the exact Trotter
    state by ~1e-5 at t = 4, since discarded components grow like sqrt(p).
    """
    wl = workloads.PARITY_L8
    T = _tebd(wl, eps_rel=1e-24)
    occ = wl.occupation()
    T.init_product(occ)
    psi = ed.dense_product(occ, wl.d)
    sched = model.step_schedule(wl.L, wl.dt)
    for k in range(1, 61):
        T.step()
        psi = ed.dense_trotter_step(psi, T.gate, sched, wl.d)
        if k % 20 == 0:
            n_d, C_d = ed.dense_observables(psi)
            assert np.max(np.abs(T.densities() - n_d)) < 1e-12
            assert np.max(np.abs(T.correlators() - C_d)) < 1e-12
            assert np.max(np.abs(T.currents() - 2 * wl.J * C_d.imag)) < 1e-12
    phi = T.full_state()
    assert abs(abs(np.vdot(phi, psi)) - 1.0) < 1e-12
    assert T.w_total < 1e-20


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_brute_force_random_small(L):
    """Random parameters and random product states vs the dense Trotterised state."""
    rng = np.random.default_rng(100 + L)
    n_max = 2
    U, J, Jnnn, K = rng.uniform(-2, 4), rng.uniform(0.5, 1.5), rng.uniform(-0.3, 0.3), rng.uniform(0, 0.2)
    jc = rng.uniform(1, L)
    dt = 0.05
    T = TEBD(L, n_max, 10 ** 6, U, J, Jnnn, K, jc, dt, w_cut=0.0, eps_rel=1e-24)
    for occ in workloads.random_product_states(L, n_max, 2, seed=L):
        T.init_product(occ)
        psi = ed.dense_product(occ, n_max + 1)
        sched = model.step_schedule(L, dt)
        for _ in range(8):
            T.step()
            psi = ed.dense_trotter_step(psi, T.gate, sched, n_max + 1)
        n_d, C_d = ed.dense_observables(psi)
        assert np.max(np.abs(T.densities() - n_d)) < 1e-12
        assert np.max(np.abs(T.correlators() - C_d)) < 1e-12


def test_largest_local_dimension_matches_dense_trotter():
    """n_max = 7 (d = 8, the library's largest; gates 512 x 512): L = 4 against the dense vector."""
    L, n_max, dt = 4, 7, 0.05
    T = TEBD(L, n_max, 10 ** 6, 2.0, 1.0, 0.15, 0.02, 2.5, dt, w_cut=0.0, eps_rel=1e-24)
    occ = np.array([3, 0, 2, 1])
    T.init_product(occ)
    psi = ed.dense_product(occ, n_max + 1)
    sched = model.step_schedule(L, dt)
    for _ in range(6):
        T.step()
        psi = ed.dense_trotter_step(psi, T.gate, sched, n_max + 1)
    n_d, C_d = ed.dense_observables(psi)
    assert np.max(np.abs(T.densities() - n_d)) < 1e-12
    assert np.max(np.abs(T.correlators() - C_d)) < 1e-12


def test_trotter_error_is_second_order():
    """Exact sector ED vs TEBD at dt and dt/2: error ratio in [3.5, 4.5] (2nd order)."""
    wl = workloads.PARITY_L8
    occ = wl.occupation()
    ex = ed.SectorED(wl.L, wl.n_max, occ, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    t_end = 1.0
    n_ex, C_ex = ex.observables(t_end)
    errs = []
    for dt in (0.04, 0.02):
        T = _tebd(wl, dt=dt)
        T.init_product(occ)
        T.step(int(round(t_end / dt)))
        errs.append(max(np.max(np.abs(T.densities() - n_ex)), np.max(np.abs(T.correlators() - C_ex))))
    ratio = errs[0] / errs[1]
    assert 3.5 <= ratio <= 4.5, (errs, ratio)
    assert errs[1] < 1e-3


def test_energy_drift_scales_as_dt2():
    """max_t |E(t) - E(0)| without truncation shrinks by ~4 when dt halves."""
    L, n_max = 6, 2
    drift = []
    for dt in (0.1, 0.05):
        T = TEBD(L, n_max, 10 ** 6, 4.0, 1.0, 0.2, 0.05, 3.5, dt, w_cut=0.0, eps_rel=1e-24)
        T.init_product(workloads.cdw(L))
        e0 = T.energy()
        m = 0.0
        for _ in range(int(round(2.0 / dt))):
            T.step()
            m = max(m, abs(T.energy() - e0))
        drift.append(m)
    ratio = drift[0] / drift[1]
    assert 3.5 <= ratio <= 4.5, (drift, ratio)


# -- free particles -------------------------------------------------------------------

def test_free_propagator_matches_bessel_bulk():
    """Exact L x L propagator of a uniform NN chain vs (1 +- J0(4t))/2 and J J1(4t)."""
    L, J = 121, 1.0
    occ = workloads.cdw(L)
    h = free.one_body_h(L, J, 0.0, 0.0, 61.0)
    c = 60  # 0-based centre site (1-based 61, odd -> occupied)
    for t in (0.3, 1.0, 2.5, 5.0):
        n, C = free.observables(free.propagator(h, t), occ)
        n_occ, n_emp, cur = free.bessel_bulk(t, J)
        assert abs(n[c] - n_occ) < 1e-12
        assert abs(n[c + 1] - n_emp) < 1e-12
        assert abs(2 * J * C[c].imag - cur) < 1e-12
        assert abs(2 * J * C[c + 1].imag + cur) < 1e-12


def test_tebd_free_bosons_trotterised():
    """U = 0, n_max >= N: TEBD == Trotterised one-body propagator (NN + NNN + trap)."""
    L, n_max, dt, steps = 8, 4, 0.02, 50
    J, Jnnn, K, jc = 1.0, 0.13, 0.02, 4.2
    occ = workloads.cdw(L)
    T = TEBD(L, n_max, 10 ** 6, 0.0, J, Jnnn, K, jc, dt, w_cut=0.0, eps_rel=1e-24)
    T.init_product(occ)
    T.step(steps)
    W = free.trotter_propagator(L, J, Jnnn, K, jc, dt, steps)
    n, C = free.observables(W, occ)
    assert np.max(np.abs(T.densities() - n)) < 1e-11
    assert np.max(np.abs(T.correlators() - C)) < 1e-11
    # and the exact (untrotterised) propagator differs only at O(dt^2)
    n_ex, _ = free.observables(free.propagator(free.one_body_h(L, J, Jnnn, K, jc), dt * steps), occ)
    assert np.max(np.abs(n - n_ex)) < 5e-3


def test_tebd_hard_core_is_free_fermions():
    """n_max = 1, J_NNN = 0, any U: TEBD == Trotterised free-fermion propagator."""
    L, dt, steps = 16, 0.02, 50
    J, K, jc = 1.0, 0.01, 8.5
    occ = workloads.cdw(L)
    T = TEBD(L, 1, 256, 7.0, J, 0.0, K, jc, dt, w_cut=0.0, eps_rel=1e-24)
    T.init_product(occ)
    T.step(steps)
    n, C = free.observables(free.trotter_propagator(L, J, 0.0, K, jc, dt, steps), occ)
    assert np.max(np.abs(T.densities() - n)) < 1e-11
    assert np.max(np.abs(T.correlators() - C)) < 1e-11


def test_two_boson_spectrum_closed_form():
    """L = 3, J_NNN = K = 0: the single three-site term is the whole of eq. (1).  In the
    two-boson sector, the states odd under reflection, (|200> - |002>)/sqrt2 and
    (|110> - |011>)/sqrt2, span an invariant block [[U, -sqrt2 J], [-sqrt2 J, 0]]: U from
    U/2 n(n-1) at n = 2, and sqrt2 J from b+ on a singly occupied site.  Its eigenvalues
    (U +- sqrt(U^2 + 8 J^2))/2, with 0 (vacuum) and 0, +-sqrt2 J (one boson, open 3-site
    chain), must all be in the spectrum.  A factor 2 on U or a missing sqrt(n) moves them."""
    rng = np.random.default_rng(3)
    for _ in range(4):
        U, J = rng.uniform(0.5, 6.0), rng.uniform(0.3, 2.0)
        for n_max in (2, 3):
            h = model.three_site_term(1, 3, n_max, U, J, 0.0, 0.0, 2.0)
            ev = np.linalg.eigvalsh(h)
            r = np.sqrt(U * U + 8 * J * J)
            for x in (0.0, np.sqrt(2) * J, -np.sqrt(2) * J, (U + r) / 2, (U - r) / 2):
                assert np.min(np.abs(ev - x)) < 1e-12, (U, J, n_max, x)
            # the vacuum and the one-boson levels fill the N <= 1 sectors exactly
            # (basis order: site 1 slowest, as the three-site term's (s1, s2, s3))
            n_tot = np.array([sum(c) for c in ed.full_basis(3, n_max)[0]])
            for N, want in ((0, [0.0]), (1, [-np.sqrt(2) * J, 0.0, np.sqrt(2) * J])):
                idx = np.flatnonzero(n_tot == N)
                assert np.allclose(np.linalg.eigvalsh(h[np.ix_(idx, idx)]), want, atol=1e-12)


def test_large_u_approaches_hard_core_as_inverse_u_squared():
    """d = 3, J_NNN = K = 0: as U grows, doubly occupied states are admixed with amplitude
    O(J/U) (Sec. III D: U -> infinity is the hard-core, free-fermion limit), so the largest
    deviation of n_j from the free-fermion values over t <= 1 falls as (J/U)^2: a factor 4
    per doubling of U.  The currents, which oscillate at frequency U, fall at the same rate
    on average (16 from U = 20 to 80).  Without the interaction the deviation would not fall
    at all; a mis-scaled one is caught by the closed-form spectrum above."""
    L, dt = 8, 0.01
    occ = workloads.cdw(L)
    h1 = free.one_body_h(L, 1.0, 0.0, 0.0, 4.5)
    dev_n, dev_c = [], []
    for U in (20.0, 40.0, 80.0):
        T = TEBD(L, 2, 256, U, 1.0, 0.0, 0.0, 4.5, dt, eps_rel=1e-14)
        T.init_product(occ)
        dn = dc = 0.0
        for k in range(1, 11):
            T.step(10)
            n, C = free.observables(free.propagator(h1, 0.1 * k), occ)
            dn = max(dn, np.max(np.abs(T.densities() - n)))
            dc = max(dc, np.max(np.abs(T.currents() - 2 * C.imag)))
        dev_n.append(dn)
        dev_c.append(dc)
    for a, b in zip(dev_n, dev_n[1:]):
        assert 3.6 < a / b < 4.4, dev_n
    assert 10.0 < dev_c[0] / dev_c[2] < 25.0, dev_c
    assert 1e-3 < dev_n[0] < 2e-2  # the hard-core limit is approached, not already reached


# -- truncation and invariants --------------------------------------------------------

def test_invariants_with_truncation():
    """chi_max = 8 forces truncation.  The contracted state keeps N exactly (the SVD
    respects U(1), Sec. II B) and norm 1 (renormalisation, Sec. II B); the canonical-form
    densities, which take the Schmidt bases as orthonormal, deviate from it only at O(w_total)."""
    L = 8
    T = TEBD(L, 3, 8, 5.0, 1.0, 0.12, 0.005, 4.5, 0.01, w_cut=1e-10, eps_rel=1e-12)
    T.init_product(workloads.cdw(L))
    T.step(150)
    assert T.w_total > 1e-6  # truncation really happened
    for lam in T.lam:
        assert abs(np.sum(lam ** 2) - 1.0) < 1e-14
    psi = T.full_state()
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12
    n_d, _ = ed.dense_observables(psi)
    assert abs(n_d.sum() - 4.0) < 1e-12
    assert abs(T.densities().sum() - 4.0) < T.w_total
    assert np.max(np.abs(T.densities() - n_d)) < T.w_total


def test_local_error_tracks_scaled_discarded_weight():
    """Observable error vs an untruncated run stays within a small multiple of w_total
    (Appendix B uses eps_local = 2 w_total / N as an error proxy)."""
    L, wl = 8, workloads.PARITY_L8
    ref = _tebd(wl, eps_rel=1e-24)
    cut = _tebd(wl, chi_max=6, eps_rel=1e-24)
    for T in (ref, cut):
        T.init_product(wl.occupation())
        T.step(100)
    err = np.max(np.abs(ref.densities() - cut.densities()))
    assert cut.w_total > 0
    assert err < 50 * cut.w_total


# -- fourth-order split (Appendix A cross-check; Suzuki's composition) ---------------

def _fourth_order_error(dt, schedule=model.step_schedule):
    """Max deviation of 4th-order TEBD from exact fixed-N ED at t = 1 (no truncation)."""
    wl = workloads.PARITY_L8
    occ = wl.occupation()
    ex = ed.SectorED(wl.L, wl.n_max, occ, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    n_ex, C_ex = ex.observables(1.0)
    T = _tebd(wl, dt=dt, eps_rel=1e-24)
    T.order = 4
    orig = model.step_schedule
    try:
        model.step_schedule = schedule
        T.init_product(occ)
        T.step(int(round(1.0 / dt)))
    finally:
        model.step_schedule = orig
    return max(np.max(np.abs(T.densities() - n_ex)), np.max(np.abs(T.correlators() - C_ex)))


def test_trotter_error_is_fourth_order():
    """Exact sector ED vs 4th-order TEBD at dt = 0.1 and 0.05: error ratio in [14, 19] (2^4 = 16)."""
    errs = [_fourth_order_error(dt) for dt in (0.1, 0.05)]
    ratio = errs[0] / errs[1]
    assert 14.0 <= ratio <= 19.0, (errs, ratio)
    assert errs[1] < 1e-6


def test_fourth_order_tebd_matches_dense_trotter():
    """The 25-layer 4th-order step on the MPS equals the same gate sequence on the dense vector."""
    L, n_max, dt = 6, 2, 0.07
    T = TEBD(L, n_max, 10 ** 6, 3.0, 1.0, 0.2, 0.05, 3.2, dt, w_cut=0.0, eps_rel=1e-24, order=4)
    occ = workloads.cdw(L)
    T.init_product(occ)
    psi = ed.dense_product(occ, n_max + 1)
    sched = model.step_schedule(L, dt, 4)
    assert len(sched) == 25 and abs(sum(tau for trip, tau in sched if trip == sched[2][0]) - dt) < 1e-15
    for _ in range(5):
        T.step()
        psi = ed.dense_trotter_step(psi, T.gate, sched, n_max + 1)
    n_d, C_d = ed.dense_observables(psi)
    assert np.max(np.abs(T.densities() - n_d)) < 1e-12
    assert np.max(np.abs(T.correlators() - C_d)) < 1e-12


def test_synthetic_saturated_state_recipe():
    """The timed input: right-canonical B_k (rows orthonormal as chi_k x d chi_{k+1}),
    sum lambda^2 = 1, bond dimensions min(chi_max, d^min(k, L-k)), seeded."""
    B, lam, chi = workloads.synthetic_state(12, 3, 20)
    assert chi == [min(20, 3 ** min(k, 12 - k)) for k in range(13)]
    for k, b in enumerate(B):
        assert b.shape == (chi[k], 3, chi[k + 1])
        M = b.reshape(chi[k], -1)
        assert np.max(np.abs(M @ M.conj().T - np.eye(chi[k]))) < 1e-12
    for x in lam:
        assert abs(np.sum(x * x) - 1.0) < 1e-14 and np.all(np.diff(x) <= 0)
    B2, lam2, _ = workloads.synthetic_state(12, 3, 20)
    assert all(np.array_equal(a, b) for a, b in zip(B, B2))


def test_oracle_records_the_closest_truncation_decision():
    """min_cut_gap: relative gap p_chi' - p_chi'+1 at the tightest cut taken."""
    T = TEBD(5, 1, 2, 1.0, 1.0, 0.0, 0.0, 3.0, 0.1)
    T.init_product(workloads.cdw(5))
    assert T.min_cut_gap == float("inf")
    T.step(3)
    assert 0.0 < T.min_cut_gap <= 1.0
