"""Pins of the U(1)-symmetric oracle (Sec. II B: U(1) symmetric tensors).

Its truncated SVDs work charge block by charge block; everything else is the
dense oracle's update.  Pinned against the dense Trotterised state vector (no
truncation), the Trotterised free-fermion propagator (hard-core bosons), the
dense oracle under truncation (the merged-spectrum reading of rule T must keep
the same chi'), and its own charge bookkeeping.
"""
import numpy as np
import pytest

from oracle import ed, free, model
from oracle.tebd import TEBD
from oracle.u1 import U1TEBD
import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _args(wl, **kw):
    a = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
             dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    a.update(kw)
    return a


def test_matches_dense_trotter_without_truncation():
    wl = workloads.PARITY_L8
    T = U1TEBD(**_args(wl, eps_rel=1e-24))
    occ = wl.occupation()
    T.init_product(occ)
    psi = ed.dense_product(occ, wl.d)
    sched = model.step_schedule(wl.L, wl.dt)
    for _ in range(40):
        T.step()
        psi = ed.dense_trotter_step(psi, T.gate, sched, wl.d)
    n_d, C_d = ed.dense_observables(psi)
    assert np.max(np.abs(T.densities() - n_d)) < 1e-12
    assert np.max(np.abs(T.correlators() - C_d)) < 1e-12
    assert abs(abs(np.vdot(T.full_state(), psi)) - 1.0) < 1e-12


def test_hard_core_is_free_fermions():
    L, dt, steps = 12, 0.02, 40
    occ = workloads.cdw(L)
    T = U1TEBD(L, 1, 256, 7.0, 1.0, 0.0, 0.01, 6.5, dt, w_cut=0.0, eps_rel=1e-24)
    T.init_product(occ)
    T.step(steps)
    n, C = free.observables(free.trotter_propagator(L, 1.0, 0.0, 0.01, 6.5, dt, steps), occ)
    assert np.max(np.abs(T.densities() - n)) < 1e-11
    assert np.max(np.abs(T.correlators() - C)) < 1e-11


def test_same_truncation_as_dense_oracle():
    """L = 32 with w_cut = 1e-10: the blocked splits keep the same chi' on every bond as the dense
    SVD and agree on the observables far inside the FP64 parity bound."""
    wl = workloads.TRUNC_L32
    u, o = U1TEBD(**_args(wl)), TEBD(**_args(wl))
    u.init_product(wl.occupation())
    o.init_product(wl.occupation())
    for _ in range(3):
        u.step(10)
        o.step(10)
        assert u.chi() == o.chi()
        assert np.max(np.abs(u.densities() - o.densities())) < 1e-12
        assert np.max(np.abs(u.currents() - o.currents())) < 1e-12
    assert abs(u.w_total - o.w_total) < 1e-15 + 1e-9 * o.w_total
    assert u.w_total > 0


def test_charge_bookkeeping():
    """Every bond label is the boson count to its left: q[0] = 0, q[L] = N, and B_k[a, s, b] vanishes
    (to rounding) unless q[k+1][b] = q[k][a] + s; the blocked reductions do a few per cent of the
    dense m^3 work."""
    wl = workloads.TRUNC_L32
    T = U1TEBD(**_args(wl))
    T.init_product(wl.occupation())
    T.step(20)
    N = int(wl.occupation().sum())
    assert T.q[0].tolist() == [0] and T.q[wl.L].tolist() == [N]
    for k in range(wl.L):
        allowed = T.q[k + 1][None, None, :] == T.q[k][:, None, None] + np.arange(wl.d)[None, :, None]
        assert np.max(np.abs(np.where(allowed, 0.0, T.B[k]))) < 1e-13, k
    assert T.block_fraction() < 0.1


def test_mutation_wrong_column_charge_is_caught(monkeypatch):
    """A planted bookkeeping mistake (the columns of the first split forget s3 in their charge)
    puts weight outside the charge blocks, which the oracle's own check refuses."""
    def bad(self, i):
        sv = np.arange(self.d)
        row_q = (self.q[i][:, None] + sv[None, :]).ravel()
        col_q = (self.q[i + 3][None, None, :] - sv[:, None, None] + 0 * sv[None, :, None]).ravel()
        return row_q, col_q
    monkeypatch.setattr(U1TEBD, "_split1_charges", bad)
    T = U1TEBD(6, 2, 64, 3.0, 1.0, 0.2, 0.05, 3.5, 0.05, eps_rel=1e-24)
    T.init_product(workloads.cdw(6))
    with pytest.raises(AssertionError, match="outside the charge blocks"):
        T.step(2)


def test_charge_labelled_synthetic_state():
    """workloads.synthetic_state_u1: right-canonical charge blocks, labels from 0 to N, and one A-layer
    update of three triples gives the same new spectra in the U(1) oracle as in the dense one."""
    L, d, chi, N = 32, 4, 256, 16
    B, lam, q = workloads.synthetic_state_u1(L, d, chi, N)
    assert q[0].tolist() == [0] and q[L].tolist() == [N]
    for k in range(L):
        M = B[k].reshape(B[k].shape[0], -1)
        assert np.max(np.abs(M @ M.conj().T - np.eye(M.shape[0]))) < 1e-12
        assert len(q[k]) <= min(chi, d ** min(k, L - k)) and np.all(np.diff(q[k]) >= 0)
        assert abs(np.sum(lam[k] ** 2) - 1.0) < 1e-14
    wl = workloads.TRUNC_L32
    u, o = U1TEBD(**_args(wl)), TEBD(**_args(wl))
    u.set_state(B, lam, q)
    o.set_state(B, lam)
    for j in (1, 13, 25):
        G = o.gate(j, wl.dt / 2)
        u.apply_gate(j - 1, G)
        o.apply_gate(j - 1, G)
        for b in (j, j + 1):
            assert len(u.lam[b]) == len(o.lam[b])
            assert np.max(np.abs(u.lam[b] - o.lam[b])) < 1e-12
    assert u.block_fraction() < 0.1


def test_mutation_per_block_truncation_is_caught(monkeypatch):
    """A planted reading mistake: rule T applied to each charge block on its own (with the block's
    own weight as the total) instead of once to the merged spectrum of the cut.  On the truncating
    L = 32 chain the blocked chi' then leaves the dense oracle's, which the pin above requires."""
    from oracle import u1 as u1mod

    def per_block(self, M, row_q, col_q):
        keep_s, keep_v, keep_q = [], [], []
        w_all = 0.0
        for c in np.unique(row_q):
            r, k = np.flatnonzero(row_q == c), np.flatnonzero(col_q == c)
            if len(k) == 0:
                continue
            _, s, Vh = u1mod.svd_desc(M[np.ix_(r, k)])
            if not np.sum(s * s) > 0.0:
                continue
            n, w = u1mod.truncation_rule(s, self.chi_max, self.w_cut, self.eps_rel)
            w_all += w
            for j in range(n):
                row = np.zeros(M.shape[1], dtype=M.dtype)
                row[k] = Vh[j]
                keep_s.append(s[j]), keep_v.append(row), keep_q.append(c)
        order = np.argsort(-np.array(keep_s), kind="stable")[: self.chi_max]
        s = np.array(keep_s)[order]
        norm = np.sqrt(np.sum(s * s))
        return s / norm, np.array(keep_v)[order], np.array(keep_q)[order], norm, w_all

    monkeypatch.setattr(U1TEBD, "_block_svd", per_block)
    wl = workloads.TRUNC_L32
    u, o = U1TEBD(**_args(wl)), TEBD(**_args(wl))
    u.init_product(wl.occupation())
    o.init_product(wl.occupation())
    u.step(10)
    o.step(10)
    assert u.chi() != o.chi()
