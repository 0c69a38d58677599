"""TEBD with U(1)-symmetric tensors (oracle), as the paper runs it (Sec. II B).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The particle number N is conserved by every gate (Sec. II B), so each bond's
Schmidt vectors can carry a definite charge: q[k][a] = the number of bosons on
sites 0..k-1 (0-based) in Schmidt vector a of bond k, with q[0] = [0] and
q[L] = [N].  B_k[a, s, b] may be non-zero only where q[k+1][b] = q[k][a] + s.

The local update is the one of ``tebd.TEBD`` (same order, same B-form
formulas); what changes is the truncated SVD.  The matrix being split,
theta' with rows (a, s1) and columns (s2, s3, b), is block diagonal in the
charge of the cut, q[i][a] + s1 = q[i+3][b] - s2 - s3, so each charge block is
decomposed on its own; the singular values of all blocks are merged, sorted
descending (ties: block order, then index), and reading T's rule picks the kept
count from the merged list.  The kept vectors take their block's charge as the
new bond label.  The second split, R = diag(s) V1^+ with rows (a', s2) and
columns (s3, b), is block diagonal in q[i+1][a'] + s2 = q[i+3][b] - s3.

Stored tensors stay dense here (only the decompositions use the blocks), so the
observables are those of the dense oracle.
"""
from __future__ import annotations

import numpy as np

from .tebd import TEBD, svd_desc, truncation_rule


class U1TEBD(TEBD):
    """Dense-storage TEBD whose truncated SVDs run block by block over U(1) charges."""

    def init_product(self, occ):
        """Product state (eq. (2) form) with its bond charges: the boson count left of each bond."""
        super().init_product(occ)
        occ = np.asarray(occ, dtype=np.int64)
        self.q = [np.array([int(occ[:k].sum())], dtype=np.int64) for k in range(self.L + 1)]
        self.block_work = [0.0, 0.0]  # [sum over splits of sum_blocks b^3, of m^3] (Gram sizes)

    def set_state(self, B, lam, q=None):
        """Install a B-form state with its bond charge labels q[k] (boson count left of bond k,
        one entry per Schmidt index); the tensors must vanish outside the allowed charges."""
        if q is None:
            raise ValueError("the U(1) oracle needs the bond charge labels")
        super().set_state(B, lam)
        self.q = [np.asarray(x, dtype=np.int64).copy() for x in q]
        for k in range(self.L):
            ok = self.q[k + 1][None, None, :] == self.q[k][:, None, None] + np.arange(self.d)[None, :, None]
            if np.any(np.where(ok, 0.0, np.abs(self.B[k])) > 0.0):
                raise ValueError(f"site {k}: entries outside the allowed charges")
        self.block_work = [0.0, 0.0]

    def _block_svd(self, M, row_q, col_q):
        """Truncated SVD of M, block diagonal in charge: returns (s normalised, Vh rows, charges,
        norm of the kept values, discarded weight)."""
        tot = float(np.sum(np.abs(M) ** 2))
        blocks = []
        inside = 0.0
        for c in np.unique(row_q):
            r = np.flatnonzero(row_q == c)
            k = np.flatnonzero(col_q == c)
            if len(k) == 0:
                continue
            Mb = M[np.ix_(r, k)]
            inside += float(np.sum(np.abs(Mb) ** 2))
            _, s, Vh = svd_desc(Mb)
            blocks.append((c, k, s, Vh))
            self.block_work[0] += float(len(r)) ** 3
        self.block_work[1] += float(M.shape[0]) ** 3
        if abs(tot - inside) > 1e-12 * max(tot, 1e-300):
            raise AssertionError("weight outside the charge blocks: the labels are inconsistent")
        # merge the spectra: descending, ties by block order then index (stable)
        entries = [(-float(s[j]), bi, j) for bi, (_, _, s, _) in enumerate(blocks) for j in range(len(s))]
        entries.sort()
        s_all = np.array([-e[0] for e in entries])
        keep, w = truncation_rule(s_all, self.chi_max, self.w_cut, self.eps_rel)
        if keep < len(s_all):
            self.min_cut_gap = min(self.min_cut_gap,
                                   float((s_all[keep - 1] ** 2 - s_all[keep] ** 2) / s_all[keep - 1] ** 2))
        s_kept = s_all[:keep]
        Vh = np.zeros((keep, M.shape[1]), dtype=M.dtype)
        charges = np.empty(keep, dtype=np.int64)
        for n, (_, bi, j) in enumerate(entries[:keep]):
            c, cols, _, Vb = blocks[bi]
            Vh[n, cols] = Vb[j]
            charges[n] = c
        norm = np.sqrt(np.sum(s_kept * s_kept))
        return s_kept / norm, Vh, charges, norm, w

    def _split1_charges(self, i: int):
        """Charge of the cut after site i for the rows (a, s1) and columns (s2, s3, b) of theta'."""
        sv = np.arange(self.d)
        row_q = (self.q[i][:, None] + sv[None, :]).ravel()
        col_q = (self.q[i + 3][None, None, :] - sv[:, None, None] - sv[None, :, None]).ravel()
        return row_q, col_q

    def _split2_charges(self, q1: np.ndarray, i: int):
        """Charge of the cut after site i+1 for the rows (a', s2) and columns (s3, b) of R."""
        sv = np.arange(self.d)
        return (q1[:, None] + sv[None, :]).ravel(), (self.q[i + 3][None, :] - sv[:, None]).ravel()

    def apply_gate(self, i: int, G: np.ndarray):
        """The update of ``TEBD.apply_gate`` with both SVDs taken by charge blocks."""
        d = self.d
        B0, B1, B2 = self.B[i], self.B[i + 1], self.B[i + 2]
        chl, chr_ = B0.shape[0], B2.shape[2]
        th = np.tensordot(np.tensordot(B0, B1, axes=(2, 0)), B2, axes=(3, 0)).reshape(chl, d ** 3, chr_)
        C = np.einsum("ps,asb->apb", G, th)
        theta = (self.lam[i][:, None, None] * C).reshape(chl * d, d * d * chr_)
        row_q, col_q = self._split1_charges(i)
        s1, V1h, q1, n1, w1 = self._block_svd(theta, row_q, col_q)
        k1 = len(s1)
        self.B[i] = (C.reshape(chl * d, d * d * chr_) @ V1h.conj().T).reshape(chl, d, k1) / n1
        self.lam[i + 1] = s1
        self.q[i + 1] = q1
        R = (s1[:, None] * V1h).reshape(k1 * d, d * chr_)
        row_q2, col_q2 = self._split2_charges(q1, i)
        s2, V2h, q2, n2, w2 = self._block_svd(R, row_q2, col_q2)
        k2 = len(s2)
        self.B[i + 1] = (V1h.reshape(k1 * d, d * chr_) @ V2h.conj().T).reshape(k1, d, k2) / n2
        self.B[i + 2] = V2h.reshape(k2, d, chr_)
        self.lam[i + 2] = s2
        self.q[i + 2] = q2
        self.w_total += w1 + w2
        return w1, w2

    def block_fraction(self) -> float:
        """sum_blocks b^3 / sum m^3 over every split so far (the eigen-solver work of a blocked
        reduction relative to the dense one, taking the Gram size b of each block)."""
        return self.block_work[0] / self.block_work[1] if self.block_work[1] else 1.0
