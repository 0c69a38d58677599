"""Super-site TEBD, the paper's own way of handling the NNN term (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. II B groups every two neighbouring sites into one super site of local
dimension d_eff = d^2, which turns the NNN chain of L sites into a
nearest-neighbour chain of L_eff = L/2 super sites; an odd chain first gets one
extra empty site at its end (the paper's 121 sites become 122, L_eff = 61).
The extra site is a site of eq. (1) like any other (hopping, trap), so the
model simulated is eq. (1) on L' = L + (L mod 2) sites.

Super site k (1-based, k = 1..L_eff) holds physical sites (2k-1, 2k); its basis
index is sigma = s_a d + s_b with s_a the occupation of site 2k-1.

Reading of the split (the paper gives no formula): every term of eq. (1) that
couples two super sites lies inside one super bond (k, k+1): the NN hop
(2k, 2k+1) and both NNN hops (2k-1, 2k+1), (2k, 2k+2).  The terms inside a
super site (its NN hop (2k-1, 2k) and the on-site terms of its two sites) are
shared equally among the one or two bonds that contain it, so that
sum_k h_k equals eq. (1) exactly.  Second-order Trotter for a NN chain
(Sec. II B): odd bonds for dt/2, even bonds for dt, odd bonds for dt/2.  One
SVD per gate; the update is the B-form two-site update of Vidal's TEBD (Sec. I).
"""
from __future__ import annotations

import numpy as np

from . import model
from .tebd import svd_desc, truncation_rule


def padded_length(L: int) -> int:
    """L' = L rounded up to even (the extra empty site of Sec. II B)."""
    return L + (L % 2)


def _op4(ops, d):
    """Kronecker product of four one-site operators (positions 0..3, position 3 fastest)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for o in ops:
        out = np.kron(out, o)
    return out


def supersite_multiplicity(k: int, L_eff: int) -> int:
    """Number of super bonds (k', k'+1), 1 <= k' <= L_eff - 1, containing super site k."""
    return int(k >= 2) + int(k <= L_eff - 1)


def bond_term(k: int, L: int, n_max: int, U: float, J: float, Jnnn: float, K: float,
              jc: float) -> np.ndarray:
    """h_k on super sites (k, k+1), 1-based k; a d^4 x d^4 matrix over physical sites
    (2k-1, 2k, 2k+1, 2k+2) in that order (site 2k+2 fastest), i.e. (sigma_k, sigma_{k+1}).

    L is the physical length before padding; eq. (1) is taken on L' = padded_length(L)."""
    Lp = padded_length(L)
    L_eff = Lp // 2
    if L_eff < 2 or not (1 <= k <= L_eff - 1):
        raise ValueError("super bonds need L_eff >= 2 and 1 <= k <= L_eff - 1")
    d = n_max + 1
    b, num, one = model.local_ops(n_max)
    bd = b.conj().T

    def on(op, pos):
        ops = [one] * 4
        ops[pos] = op
        return _op4(ops, d)

    def hop(p, q):  # b+_p b_q + h.c. on positions p != q
        ops = [one] * 4
        ops[p] = bd
        ops[q] = b
        t = _op4(ops, d)
        return t + t.conj().T

    # couplings between the two super sites: each belongs to this bond only
    h = -J * hop(1, 2) - Jnnn * (hop(0, 2) + hop(1, 3))
    # terms inside super site k (positions 0, 1) and k+1 (positions 2, 3), shared
    for kk, (p0, p1) in ((k, (0, 1)), (k + 1, (2, 3))):
        c = supersite_multiplicity(kk, L_eff)
        inner = -J * hop(p0, p1)
        for pos, site in ((p0, 2 * kk - 1), (p1, 2 * kk)):
            inner = inner + on(0.5 * U * (num @ (num - one)) + 0.5 * K * (site - jc) ** 2 * num, pos)
        h = h + inner / c
    return h


def step_schedule(L_eff: int, dt: float):
    """[(bonds, tau), ...] of one second-order step: odd bonds dt/2, even bonds dt, odd bonds dt/2
    (1-based bond k joins super sites k and k+1; bonds of one layer share no super site)."""
    odd = [k for k in range(1, L_eff) if k % 2 == 1]
    even = [k for k in range(1, L_eff) if k % 2 == 0]
    out = [(odd, dt / 2)]
    if even:
        out.append((even, dt))
    out.append((odd, dt / 2))
    return out


class SuperSiteTEBD:
    """Plain FP64 super-site TEBD for eq. (1) (oracle).

    Same parameters as the three-site oracle; L is the physical length (padded
    to even internally).  Observables are reported for the L' = padded_length(L)
    physical sites; the padded site is the last one.
    """

    def __init__(self, L, n_max, chi_max, U, J, Jnnn, K, jc, dt, w_cut=0.0, eps_rel=1e-12):
        if L < 3:
            raise ValueError("L >= 3 required")
        self.L, self.Lp = L, padded_length(L)
        self.L_eff = self.Lp // 2
        self.n_max, self.d = n_max, n_max + 1
        self.de = self.d ** 2
        self.chi_max, self.dt = chi_max, dt
        self.U, self.J, self.Jnnn, self.K, self.jc = U, J, Jnnn, K, jc
        self.w_cut, self.eps_rel = w_cut, eps_rel
        self.h = [bond_term(k, L, n_max, U, J, Jnnn, K, jc) for k in range(1, self.L_eff)]
        self._gates = {}
        self.B = None
        self.lam = None
        self.t, self.steps, self.w_total = 0.0, 0, 0.0

    def gate(self, k: int, tau: float) -> np.ndarray:
        """exp(-i h_k tau) of super bond k (1-based), built once and cached (Sec. II B)."""
        key = (k, tau)
        if key not in self._gates:
            self._gates[key] = model.gate(self.h[k - 1], tau)
        return self._gates[key]

    def init_product(self, occ):
        """Product state over the L physical sites (the padded site starts empty)."""
        occ = np.asarray(occ)
        if occ.shape != (self.L,) or occ.min() < 0 or occ.max() > self.n_max:
            raise ValueError("occupation vector out of range")
        full = np.zeros(self.Lp, dtype=np.int64)
        full[:self.L] = occ
        self.B = []
        for k in range(self.L_eff):
            t = np.zeros((1, self.de, 1), dtype=np.complex128)
            t[0, int(full[2 * k]) * self.d + int(full[2 * k + 1]), 0] = 1.0
            self.B.append(t)
        self.lam = [np.ones(1) for _ in range(self.L_eff + 1)]
        self.t, self.steps, self.w_total = 0.0, 0, 0.0

    def chi(self):
        """Bond dimensions of the super-site chain, bonds 0..L_eff."""
        return [len(x) for x in self.lam]

    def apply_gate(self, i: int, G: np.ndarray):
        """Two-site update of super sites (i, i+1), 0-based:
        theta~ = B_i B_{i+1}; C = G theta~; theta' = lam[i] (.) C; SVD of theta' as
        (chi_l d_eff) x (d_eff chi_r), truncate (reading T), renormalise;
        B_i = C V^+ / ||s||, B_{i+1} = V^+ rows, lam[i+1] = s / ||s||."""
        de = self.de
        B0, B1 = self.B[i], self.B[i + 1]
        chl, chr_ = B0.shape[0], B1.shape[2]
        th = np.tensordot(B0, B1, axes=(2, 0)).reshape(chl, de * de, chr_)
        C = np.einsum("ps,asb->apb", G, th)
        theta = (self.lam[i][:, None, None] * C).reshape(chl * de, de * chr_)
        _, s, Vh = svd_desc(theta)
        k, w = truncation_rule(s, self.chi_max, self.w_cut, self.eps_rel)
        s, Vh = s[:k], Vh[:k]
        norm = np.sqrt(np.sum(s * s))
        self.B[i] = (C.reshape(chl * de, de * chr_) @ Vh.conj().T).reshape(chl, de, k) / norm
        self.B[i + 1] = Vh.reshape(k, de, chr_)
        self.lam[i + 1] = s / norm
        self.w_total += w
        return w

    def step(self, n: int = 1):
        """n second-order steps of the NN split (odd bonds dt/2, even dt, odd dt/2)."""
        sched = step_schedule(self.L_eff, self.dt)
        for _ in range(n):
            for bonds, tau in sched:
                for k in bonds:
                    self.apply_gate(k - 1, self.gate(k, tau))
            self.steps += 1
            self.t = self.steps * self.dt

    # -- observables (eqs. (5), (8), canonical form) ----------------------------
    def _site_ops(self):
        """b, b^+, n and 1 on one physical site (truncated Fock space, Sec. II B)."""
        b, num, one = model.local_ops(self.n_max)
        return b, b.conj().T, num, one

    def densities(self) -> np.ndarray:
        """n_j for the L' physical sites: n of position a or b of super site (j+1)//2."""
        _, _, num, one = self._site_ops()
        na, nb = np.kron(num, one), np.kron(one, num)
        out = np.empty(self.Lp)
        for k in range(self.L_eff):
            rho = np.einsum("a,asb,atb->st", self.lam[k] ** 2, self.B[k].conj(), self.B[k])
            out[2 * k] = np.real(np.trace(rho @ na.T))
            out[2 * k + 1] = np.real(np.trace(rho @ nb.T))
        return out

    def correlators(self) -> np.ndarray:
        """C_j = <b+_j b_{j+1}> for the L' - 1 physical NN bonds: inside a super site
        (j odd) a one-super-site expectation, across two (j even) a two-super-site one."""
        b, bd, _, one = self._site_ops()
        inner = np.kron(bd, b)                       # b+_(2k-1) b_(2k)
        left, right = np.kron(one, bd), np.kron(b, one)  # b+ on position b of k, b on a of k+1
        out = np.empty(self.Lp - 1, dtype=np.complex128)
        for k in range(self.L_eff):
            th = self.lam[k][:, None, None] * self.B[k]
            out[2 * k] = np.vdot(th, np.einsum("st,atb->asb", inner, th))
            if k + 1 < self.L_eff:
                th2 = np.tensordot(th, self.B[k + 1], axes=(2, 0))
                out[2 * k + 1] = np.vdot(th2, np.einsum("su,tv,auvb->astb", left, right, th2))
        return out

    def currents(self) -> np.ndarray:
        """2 J Im C_j (reading C)."""
        return 2.0 * self.J * np.imag(self.correlators())

    def full_state(self) -> np.ndarray:
        """Dense state over the L' physical sites, shape (d,)*L' (small chains only)."""
        psi = (self.lam[0][:, None, None] * self.B[0]).reshape(self.de, -1)
        for k in range(1, self.L_eff):
            psi = np.tensordot(psi, self.B[k], axes=(-1, 0)).reshape(-1, self.B[k].shape[2])
        return psi.reshape((self.d,) * self.Lp)
