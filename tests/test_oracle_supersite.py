"""Pins of the super-site oracle (Sec. II B's grouping of site pairs) against what
the paper and the mathematics fix, independently of the three-site oracle.

* the bond terms sum to eq. (1) assembled directly in the Fock basis (on the
  chain padded to even length with one empty site, as Sec. II B does);
* without truncation the MPS run equals the dense state vector evolved by the
  same gates (isolates the MPS machinery and the observables);
* against exact fixed-N ED the error is second order in dt;
* at U = 0 with enough n_max (free bosons) and at n_max = 1, J_NNN = 0
  (hard-core bosons = free fermions) it equals the Trotterised one-body
  propagator of the same split;
* the paper's flanked CDW on a short odd chain converges to exact ED.
"""
import numpy as np
import pytest

from oracle import ed, free, supersite
from oracle.supersite import SuperSiteTEBD
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _apply_block(psi, G, i, width, d):
    """G (d^width x d^width) on physical sites i..i+width-1 (0-based) of psi[(d,)*L]."""
    L = psi.ndim
    axes = tuple(range(i, i + width))
    x = np.moveaxis(psi, axes, tuple(range(width))).reshape(d ** width, -1)
    rest = tuple(np.delete(psi.shape, axes))
    x = (G @ x).reshape((d,) * width + rest)
    return np.moveaxis(x, tuple(range(width)), axes).reshape((d,) * L)


def _dense_step(psi, T, d):
    for bonds, tau in supersite.step_schedule(T.L_eff, T.dt):
        for k in bonds:
            psi = _apply_block(psi, T.gate(k, tau), 2 * k - 2, 4, d)
    return psi


@pytest.mark.parametrize("L,n_max", [(4, 2), (5, 2), (6, 2), (7, 1), (8, 1)])
def test_bond_terms_sum_to_eq1(L, n_max):
    """sum_k h_k = eq. (1) on L' = L + (L mod 2) sites, built in the Fock basis."""
    rng = np.random.default_rng(10 + L)
    U, J, Jnnn, K = rng.uniform(0.5, 3, size=4)
    jc = (L + 1) / 2 + 0.2
    Lp = supersite.padded_length(L)
    d = n_max + 1
    basis, index = ed.full_basis(Lp, n_max)
    H = ed.hamiltonian(basis, index, Lp, n_max, U, J, -Jnnn, K, jc)
    S = np.zeros_like(H)
    for k in range(1, Lp // 2):
        h = supersite.bond_term(k, L, n_max, U, J, -Jnnn, K, jc)
        S += np.kron(np.kron(np.eye(d ** (2 * k - 2)), h), np.eye(d ** (Lp - 2 * k - 2)))
    assert np.max(np.abs(S - H)) < 1e-13


def test_paper_sizes():
    """Sec. II C: 121 sites plus one empty site give L_eff = 61 super sites of d_eff = 25 (n_max = 4)."""
    assert supersite.padded_length(121) // 2 == 61
    T = SuperSiteTEBD(121, 4, 40, 2.442, 1.0, -0.12, 0.01, 61.0, 0.05 * np.pi / 2)
    assert (T.L_eff, T.de, len(T.h)) == (61, 25, 60)


def test_schedule_gives_every_bond_dt_and_disjoint_layers():
    for L_eff in (2, 3, 6, 61):
        tot = {}
        for bonds, tau in supersite.step_schedule(L_eff, 0.02):
            sites = [s for k in bonds for s in (k, k + 1)]
            assert len(sites) == len(set(sites))
            for k in bonds:
                tot[k] = tot.get(k, 0.0) + tau
        assert sorted(tot) == list(range(1, L_eff)) and all(abs(v - 0.02) < 1e-15 for v in tot.values())


@pytest.mark.parametrize("L,seed", [(5, 0), (6, 1), (6, 2)])
def test_matches_dense_trotter(L, seed):
    """No truncation: the MPS run equals the dense vector evolved by the same gates."""
    rng = np.random.default_rng(seed)
    n_max, d = 2, 3
    U, J, Jnnn, K = rng.uniform(-2, 4), rng.uniform(0.5, 1.5), rng.uniform(-0.3, 0.3), rng.uniform(0, 0.2)
    jc = rng.uniform(1, L)
    T = SuperSiteTEBD(L, n_max, 10 ** 6, U, J, Jnnn, K, jc, 0.05, w_cut=0.0, eps_rel=1e-24)
    occ = workloads.random_product_states(L, n_max, 1, seed=seed)[0]
    T.init_product(occ)
    psi = ed.dense_product(list(occ) + [0] * (T.Lp - L), d)
    for _ in range(8):
        T.step()
        psi = _dense_step(psi, T, d)
    n_d, C_d = ed.dense_observables(psi)
    assert np.max(np.abs(T.densities() - n_d)) < 1e-12
    assert np.max(np.abs(T.correlators() - C_d)) < 1e-12
    assert abs(abs(np.vdot(T.full_state(), psi)) - 1.0) < 1e-12
    assert T.w_total < 1e-20


def test_trotter_error_is_second_order():
    """Exact sector ED on L = 8 (d = 4, N = 4) vs the super-site run at dt and dt/2."""
    wl = workloads.PARITY_L8
    occ = wl.occupation()
    ex = ed.SectorED(wl.L, wl.n_max, occ, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    n_ex, C_ex = ex.observables(1.0)
    errs = []
    for dt in (0.04, 0.02):
        T = SuperSiteTEBD(wl.L, wl.n_max, 256, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, dt, eps_rel=1e-24)
        T.init_product(occ)
        T.step(int(round(1.0 / dt)))
        errs.append(max(np.max(np.abs(T.densities() - n_ex)), np.max(np.abs(T.correlators() - C_ex))))
    assert 3.5 <= errs[0] / errs[1] <= 4.5, errs
    assert errs[1] < 1e-3


def test_free_bosons_trotterised():
    """U = 0, n_max >= N: the run equals the Trotterised one-body propagator of the
    super-site split (NN, NNN and trap), odd L padded with an empty site."""
    L, N = 7, 2
    occ = np.zeros(L, dtype=np.int64)
    occ[[2, 4]] = 1
    J, Jnnn, K, jc, dt, steps = 1.0, 0.3, 0.05, 3.7, 0.05, 12
    T = SuperSiteTEBD(L, N, 10 ** 6, 0.0, J, Jnnn, K, jc, dt, w_cut=0.0, eps_rel=1e-24)
    T.init_product(occ)
    T.step(steps)
    W = free.supersite_trotter_propagator(T.Lp, J, Jnnn, K, jc, dt, steps)
    n, C = free.observables(W, np.concatenate([occ, [0]]))
    assert np.max(np.abs(T.densities() - n)) < 1e-11
    assert np.max(np.abs(T.correlators() - C)) < 1e-11


def test_hard_core_is_free_fermions():
    """n_max = 1, J_NNN = 0, any U: the run equals the same one-body propagator."""
    L, dt, steps = 12, 0.02, 40
    J, K, jc = 1.0, 0.01, 6.5
    occ = workloads.cdw(L)
    T = SuperSiteTEBD(L, 1, 256, 7.0, J, 0.0, K, jc, dt, w_cut=0.0, eps_rel=1e-24)
    T.init_product(occ)
    T.step(steps)
    n, C = free.observables(free.supersite_trotter_propagator(L, J, 0.0, K, jc, dt, steps), occ)
    assert np.max(np.abs(T.densities() - n)) < 1e-11
    assert np.max(np.abs(T.correlators() - C)) < 1e-11


def test_flanked_cdw_converges_to_exact_ed():
    """The paper's initial-state form on a short odd chain: L = 11 (padded to 12),
    3 bosons in the middle, Table Ib set a; exact fixed-N ED on the 12 sites.
    The error, the padded site included, falls by ~4 when dt halves."""
    L, N = 11, 3
    U, Jnnn, K = workloads.PAPER_PARAMS["a"]
    jc = (L + 1) / 2
    occ = workloads.flanked_cdw(L, N)
    Lp = supersite.padded_length(L)
    occ_p = tuple(int(x) for x in np.concatenate([occ, [0]]))
    ex = ed.SectorED(Lp, 3, occ_p, U, 1.0, Jnnn, K, jc)
    n_ex, C_ex = ex.observables(1.0)
    errs = []
    for dt in (0.05, 0.025):
        T = SuperSiteTEBD(L, 3, 10 ** 6, U, 1.0, Jnnn, K, jc, dt, eps_rel=1e-24)
        T.init_product(occ)
        T.step(int(round(1.0 / dt)))
        n = T.densities()
        errs.append(max(np.max(np.abs(n - n_ex)), np.max(np.abs(T.correlators() - C_ex))))
        assert abs(n.sum() - N) < 1e-10
    assert 3.5 <= errs[0] / errs[1] <= 4.5, errs


def test_invariants_with_truncation():
    """chi_max = 6 forces truncation.  The contracted state keeps N exactly (the SVD respects
    U(1)) and norm 1 (renormalisation); the canonical-form densities, which assume
    orthonormality (Sec. II B), deviate from it only at O(w_total)."""
    T = SuperSiteTEBD(10, 3, 6, 5.0, 1.0, 0.12, 0.005, 5.5, 0.02, w_cut=1e-10, eps_rel=1e-12)
    T.init_product(workloads.cdw(10))
    T.step(40)
    assert T.w_total > 1e-6 and max(T.chi()) == 6
    assert all(abs(np.sum(l ** 2) - 1.0) < 1e-13 for l in T.lam)
    psi = T.full_state()
    assert abs(np.vdot(psi, psi).real - 1.0) < 1e-12
    n_d, _ = ed.dense_observables(psi)
    assert abs(n_d.sum() - 5.0) < 1e-12
    assert np.max(np.abs(T.densities() - n_d)) < T.w_total


# -- planted mistakes: each must fail one of the pins above -------------------------

def _split_error(L=6, n_max=2):
    U, J, Jnnn, K, jc = 2.0, 1.0, 0.3, 0.1, 3.3
    Lp, d = supersite.padded_length(L), n_max + 1
    basis, index = ed.full_basis(Lp, n_max)
    H = ed.hamiltonian(basis, index, Lp, n_max, U, J, Jnnn, K, jc)
    S = sum(np.kron(np.kron(np.eye(d ** (2 * k - 2)), supersite.bond_term(k, L, n_max, U, J, Jnnn, K, jc)),
                    np.eye(d ** (Lp - 2 * k - 2))) for k in range(1, Lp // 2))
    return np.max(np.abs(S - H))


def test_mutation_unshared_inner_terms(monkeypatch):
    assert _split_error() < 1e-13
    monkeypatch.setattr(supersite, "supersite_multiplicity", lambda k, L_eff: 1)
    assert _split_error() > 1e-2


def test_mutation_dropped_cross_nnn_hop(monkeypatch):
    """The NNN hop (2k, 2k+2) across each bond left out of the bond term."""
    orig = supersite.bond_term

    def bad(k, L, n_max, U, J, Jnnn, K, jc):
        b, _, one = supersite.model.local_ops(n_max)
        t = np.kron(np.kron(np.kron(one, b.conj().T), one), b)  # b+ on position 1, b on 3
        return orig(k, L, n_max, U, J, Jnnn, K, jc) + Jnnn * (t + t.conj().T)
    assert _split_error() < 1e-13
    monkeypatch.setattr(supersite, "bond_term", bad)
    assert _split_error() > 1e-2


def test_mutation_first_order_schedule(monkeypatch):
    def first_order(L_eff, dt):
        return [([k for k in range(1, L_eff) if k % 2 == 1], dt), ([k for k in range(1, L_eff) if k % 2 == 0], dt)]
    monkeypatch.setattr(supersite, "step_schedule", first_order)
    wl = workloads.PARITY_L8
    ex = ed.SectorED(wl.L, wl.n_max, wl.occupation(), wl.U, wl.J, wl.Jnnn, wl.K, wl.jc)
    n_ex, _ = ex.observables(0.5)
    errs = []
    for dt in (0.05, 0.025):
        T = SuperSiteTEBD(wl.L, wl.n_max, 256, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, dt, eps_rel=1e-24)
        T.init_product(wl.occupation())
        T.step(int(round(0.5 / dt)))
        errs.append(np.max(np.abs(T.densities() - n_ex)))
    assert not (3.5 <= errs[0] / errs[1] <= 4.5), errs


def test_mutation_swapped_positions_in_densities():
    class Bad(SuperSiteTEBD):
        def densities(self):
            return super().densities().reshape(-1, 2)[:, ::-1].reshape(-1)
    T = Bad(6, 2, 10 ** 6, 3.0, 1.0, 0.2, 0.05, 3.2, 0.05, eps_rel=1e-24)
    occ = np.array([2, 0, 1, 0, 0, 1])
    T.init_product(occ)
    psi = ed.dense_product(occ, 3)
    for _ in range(3):
        T.step()
        psi = _dense_step(psi, T, 3)
    n_d, _ = ed.dense_observables(psi)
    assert np.max(np.abs(T.densities() - n_d)) > 1e-2
