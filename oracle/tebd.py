"""Second-order TEBD on a Vidal Gamma-lambda MPS, stored in B-form (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

State (Vidal's TEBD, named in Sec. I; Sec. II B): B_k = Gamma_k lambda_k (right
canonical) for sites k = 0..L-1 (0-based here), shape (chi_left, d, chi_right),
and bond vectors lam[k] for k = 0..L, lam[k] sitting to the left of site k
(lam[0] = lam[L] = [1]).

Local update of the triple (i, i+1, i+2) with gate G (three sites where a NNN
term acts), taken in the order the method states:

  1. theta~ = B_i B_{i+1} B_{i+2}                    (contract shared bonds)
  2. C = G theta~ over the physical index sigma = (s1,s2,s3)
  3. theta' = lam[i] (.) C                           (row scaling)
  4. SVD of theta' as (chi_l d) x (d^2 chi_r); truncate (reading T);
     renormalise the kept values (reading R; Sec. II B)
  5. B_i = C V1 / ||s||   (division-free form), lam[i+1] = s / ||s||
  6. R = diag(lam[i+1]) V1^+ as (chi' d) x (d chi_r); SVD, truncate, renormalise
  7. B_{i+1} = V1^+ V2 / ||s2||,  B_{i+2} = V2^+,  lam[i+2] = s2 / ||s2||

Observables (Sec. II C, eqs. (5), (8)) are evaluated from the canonical form,
taking the Schmidt bases as orthonormal without a full contraction (Sec. II B),
after every full step (reading O).
"""
from __future__ import annotations

import numpy as np

from . import model


def truncation_rule(s: np.ndarray, chi_max: int, w_cut: float, eps_rel: float):
    """Kept count chi' and discarded weight w for descending singular values s.

    Reading T of the tolerances of Sec. II B (w_max, eps): with
    p_k = s_k^2 / sum s^2,
      chi_w   = smallest k >= 1 with sum_{i>k} p_i <= w_cut,
      chi_eps = #{k : p_k > eps_rel}  (at least 1),
      chi'    = max(1, min(chi_max, chi_w, chi_eps)),
      w       = sum_{i>chi'} p_i.
    The kept count is decided by this rule alone (never widened to a multiplet).
    """
    s = np.asarray(s, dtype=np.float64)
    p = s * s
    total = p.sum()
    if total <= 0.0:
        raise ValueError("zero matrix in truncated SVD")
    p = p / total
    tail = np.concatenate([np.cumsum(p[::-1])[::-1][1:], [0.0]])  # tail[k-1] = sum_{i>k}
    chi_w = int(np.argmax(tail <= w_cut)) + 1 if np.any(tail <= w_cut) else len(p)
    chi_eps = max(1, int(np.count_nonzero(p > eps_rel)))
    chi = max(1, min(chi_max, chi_w, chi_eps, len(p)))
    w = float(p[chi:].sum())
    return chi, w


def svd_desc(M: np.ndarray):
    """Thin SVD with descending singular values (LAPACK gesdd, gesvd fallback)."""
    try:
        U, s, Vh = np.linalg.svd(M, full_matrices=False)
    except np.linalg.LinAlgError:  # pragma: no cover - LAPACK fallback
        import scipy.linalg
        U, s, Vh = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
    return U, s, Vh


class TEBD:
    """Plain FP64 TEBD for eq. (1) with three-site gates (oracle).

    Parameters follow the library's create call: L sites, n_max (d = n_max+1),
    chi_max, U, J, J_NNN, K, j_c (1-based site coordinate), dt (hbar = J = 1
    units of Sec. I A); w_cut and eps_rel are reading T's tolerances.
    """

    def __init__(self, L, n_max, chi_max, U, J, Jnnn, K, jc, dt, w_cut=0.0, eps_rel=1e-12, order=2):
        if L < 3:
            raise ValueError("L >= 3 required (three-site gates)")
        self.L, self.n_max, self.d = L, n_max, n_max + 1
        self.chi_max, self.dt = chi_max, dt
        self.U, self.J, self.Jnnn, self.K, self.jc = U, J, Jnnn, K, jc
        self.w_cut, self.eps_rel = w_cut, eps_rel
        self.order = order
        self.h = [model.three_site_term(j, L, n_max, U, J, Jnnn, K, jc) for j in range(1, L - 1)]
        self._gates = {}
        self.B = None
        self.lam = None
        self.t = 0.0
        self.steps = 0
        self.w_total = 0.0
        self.min_cut_gap = float("inf")  # smallest (p_{chi'} - p_{chi'+1}) / p_{chi'} seen at a cut

    # -- gates -----------------------------------------------------------------
    def gate(self, j: int, tau: float) -> np.ndarray:
        """Gate of triple j (1-based) for time tau, built once and cached."""
        key = (j, tau)
        if key not in self._gates:
            self._gates[key] = model.gate(self.h[j - 1], tau)
        return self._gates[key]

    # -- state -----------------------------------------------------------------
    def init_product(self, occ):
        """Product state |occ_1, ..., occ_L> (eq. (2) form; reading I) as chi = 1 MPS."""
        occ = np.asarray(occ)
        if occ.shape != (self.L,) or occ.min() < 0 or occ.max() > self.n_max:
            raise ValueError("occupation vector out of range")
        d = self.d
        self.B = []
        for k in range(self.L):
            t = np.zeros((1, d, 1), dtype=np.complex128)
            t[0, int(occ[k]), 0] = 1.0
            self.B.append(t)
        self.lam = [np.ones(1) for _ in range(self.L + 1)]
        self.t, self.steps, self.w_total = 0.0, 0, 0.0

    def set_state(self, B, lam):
        """Install an arbitrary B-form state (used for synthetic saturated states)."""
        self.B = [np.array(b, dtype=np.complex128) for b in B]
        self.lam = [np.array(x, dtype=np.float64) for x in lam]

    def chi(self):
        """Bond dimensions chi_0..chi_L."""
        return [len(x) for x in self.lam]

    # -- local update ----------------------------------------------------------
    def _truncated_svd(self, M):
        """SVD of M, cut by reading T and renormalised (reading R); returns (s, Vh, ||s_kept||, w)."""
        U, s, Vh = svd_desc(M)
        k, w = truncation_rule(s, self.chi_max, self.w_cut, self.eps_rel)
        if k < len(s):  # record how close the decision was: relative gap at the cut
            self.min_cut_gap = min(self.min_cut_gap, float((s[k - 1] ** 2 - s[k] ** 2) / s[k - 1] ** 2))
        s = s[:k]
        norm = np.sqrt(np.sum(s * s))
        return s / norm, Vh[:k], norm, w

    def apply_gate(self, i: int, G: np.ndarray):
        """Local update of the triple (i, i+1, i+2), 0-based i (steps 1-7 above)."""
        d = self.d
        B0, B1, B2 = self.B[i], self.B[i + 1], self.B[i + 2]
        chl, chr_ = B0.shape[0], B2.shape[2]
        th = np.tensordot(np.tensordot(B0, B1, axes=(2, 0)), B2, axes=(3, 0))
        th = th.reshape(chl, d ** 3, chr_)
        C = np.einsum("ps,asb->apb", G, th)
        theta = self.lam[i][:, None, None] * C
        s1, V1h, n1, w1 = self._truncated_svd(theta.reshape(chl * d, d * d * chr_))
        k1 = len(s1)
        self.B[i] = (C.reshape(chl * d, d * d * chr_) @ V1h.conj().T).reshape(chl, d, k1) / n1
        self.lam[i + 1] = s1
        R = (s1[:, None] * V1h).reshape(k1 * d, d * chr_)
        s2, V2h, n2, w2 = self._truncated_svd(R)
        k2 = len(s2)
        self.B[i + 1] = (V1h.reshape(k1 * d, d * chr_) @ V2h.conj().T).reshape(k1, d, k2) / n2
        self.B[i + 2] = V2h.reshape(k2, d, chr_)
        self.lam[i + 2] = s2
        self.w_total += w1 + w2
        return w1, w2

    def layer(self, triples, tau):
        """One Trotter layer: the gates of the given (disjoint) triples for time tau."""
        for j in triples:
            self.apply_gate(j - 1, self.gate(j, tau))

    def step(self, n: int = 1):
        """n full steps of the Trotter split of the given order (model.step_schedule)."""
        sched = (model.step_schedule(self.L, self.dt) if self.order == 2
                 else model.step_schedule(self.L, self.dt, self.order))
        for _ in range(n):
            for triples, tau in sched:
                self.layer(triples, tau)
            self.steps += 1
            self.t = self.steps * self.dt

    # -- observables -----------------------------------------------------------
    def densities(self) -> np.ndarray:
        """n_j = sum lam[j]_a^2 |B_j[a,s,b]|^2 s  (eq. (8) in canonical form)."""
        out = np.empty(self.L)
        svals = np.arange(self.d, dtype=np.float64)
        for k in range(self.L):
            w = (self.lam[k] ** 2)[:, None, None] * np.abs(self.B[k]) ** 2
            out[k] = np.sum(w.sum(axis=(0, 2)) * svals)
        return out

    def correlators(self) -> np.ndarray:
        """C_j = <b+_j b_{j+1}> (eq. (5)) for j = 1..L-1 from theta2 = lam (.) B_j B_{j+1}."""
        b, _, _ = model.local_ops(self.n_max)
        bd = b.conj().T
        out = np.empty(self.L - 1, dtype=np.complex128)
        for k in range(self.L - 1):
            th = np.tensordot(self.B[k], self.B[k + 1], axes=(2, 0))
            th = self.lam[k][:, None, None, None] * th
            Oth = np.einsum("su,tv,auvb->astb", bd, b, th)
            out[k] = np.vdot(th, Oth)
        return out

    def currents(self) -> np.ndarray:
        """current_j = -iJ <b+_j b_{j+1} - h.c.> = 2 J Im C_j (reading C; positive = j -> j+1)."""
        return 2.0 * self.J * np.imag(self.correlators())

    def energy(self) -> float:
        """<H> = sum_j <h_j> from three-site canonical-form reduced states (oracle-only)."""
        d = self.d
        e = 0.0
        for i in range(self.L - 2):
            th = np.tensordot(np.tensordot(self.B[i], self.B[i + 1], axes=(2, 0)), self.B[i + 2], axes=(3, 0))
            th = (self.lam[i][:, None, None, None, None] * th)
            chl, chr_ = th.shape[0], th.shape[-1]
            th = th.reshape(chl, d ** 3, chr_)
            e += np.real(np.vdot(th, np.einsum("ps,asb->apb", self.h[i], th)))
        return float(e)

    def full_state(self) -> np.ndarray:
        """Dense state vector of shape (d,)*L by full contraction (small L only)."""
        psi = self.lam[0][:, None, None] * self.B[0]  # (1, d, chi)
        psi = psi.reshape(self.d, -1)
        for k in range(1, self.L):
            psi = np.tensordot(psi, self.B[k], axes=(-1, 0))
            psi = psi.reshape(-1, self.B[k].shape[2])
        return psi.reshape((self.d,) * self.L)
