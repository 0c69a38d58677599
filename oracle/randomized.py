"""Truncation by a randomized range finder (oracle), the cheaper SVD the paper
points to for larger bond dimensions (Sec. V: reduced-rank randomized SVD in
TEBD, after Tamascelli et al. 2015).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For an m x n matrix M whose leading k singular triplets are wanted, the
published randomized SVD (Halko, Martinsson and Tropp, SIAM Review 53, 2011,
Algorithms 4.3/4.4 and 5.1) takes, with a sketch of l = k + p columns:

  1. Y = M Omega with an n x l Gaussian test matrix Omega;
  2. q power iterations, each re-orthonormalised: Q = qr(Y), Z = qr(M^+ Q),
     Y = M Z (they sharpen the sketch when the spectrum decays slowly);
  3. Q = qr(Y), an orthonormal basis of the sampled range;
  4. the small matrix C = Q^+ M (l x n) and its exact SVD C = U~ S V^+;
  5. U = Q U~; the singular triplets of M are approximated by (U, S, V).

Every product in it is a dense GEMM, and the only decomposition left is of an
l x n matrix, which is why it suits tensor cores.  The random numbers are an
input: ``omega`` is passed in (here from ``workloads``), never drawn inside.

Truncation keeps reading T, written for a partial spectrum: p_i = s_i^2 / t
with t = ||M||_F^2 (known exactly), the tail after k' kept values is
t - sum_{i<=k'} s_i^2, and chi_eps counts the sketched values above eps_rel.
"""
from __future__ import annotations

import numpy as np

from .tebd import TEBD


def randomized_svd(M: np.ndarray, omega: np.ndarray, q: int = 2):
    """(U, s, Vh) of rank l = omega.shape[1] from the range finder above (steps 1-5)."""
    Y = M @ omega
    for _ in range(q):
        Q, _ = np.linalg.qr(Y)
        Z, _ = np.linalg.qr(M.conj().T @ Q)
        Y = M @ Z
    Q, _ = np.linalg.qr(Y)
    C = Q.conj().T @ M
    Ut, s, Vh = np.linalg.svd(C, full_matrices=False)
    return Q @ Ut, s, Vh


def truncation_rule_partial(s: np.ndarray, total: float, chi_max: int, w_cut: float, eps_rel: float):
    """Reading T on the leading values s (descending) of a matrix with ||M||_F^2 = total."""
    p = (np.asarray(s, dtype=np.float64) ** 2) / total
    kept = np.cumsum(p)
    tail = np.maximum(1.0 - kept, 0.0)  # tail after keeping 1, 2, ... values
    ok = np.flatnonzero(tail <= w_cut)
    chi_w = int(ok[0]) + 1 if len(ok) else len(p)
    chi_eps = max(1, int(np.count_nonzero(p > eps_rel)))
    chi = max(1, min(chi_max, chi_w, chi_eps, len(p)))
    return chi, float(max(1.0 - kept[chi - 1], 0.0))


class RandomizedTEBD(TEBD):
    """The dense oracle's update with each truncated SVD taken by the range finder.

    omega_fn(n, l, call) returns the n x l complex Gaussian test matrix of the
    call-th decomposition (an input); oversample p and power iterations q set the
    sketch l = min(chi_max + p, m, n)."""

    def __init__(self, *args, omega_fn=None, oversample: int = 10, power_iters: int = 2, **kw):
        super().__init__(*args, **kw)
        if omega_fn is None:
            raise ValueError("the test matrices are an input (omega_fn)")
        self.omega_fn, self.oversample, self.power_iters = omega_fn, oversample, power_iters
        self.calls = 0

    def _truncated_svd(self, M):
        m, n = M.shape
        l = min(self.chi_max + self.oversample, m, n)
        omega = self.omega_fn(n, l, self.calls)
        self.calls += 1
        _, s, Vh = randomized_svd(M, omega, self.power_iters)
        total = float(np.sum(np.abs(M) ** 2))
        k, w = truncation_rule_partial(s, total, self.chi_max, self.w_cut, self.eps_rel)
        if k < len(s):
            self.min_cut_gap = min(self.min_cut_gap, float((s[k - 1] ** 2 - s[k] ** 2) / s[k - 1] ** 2))
        s = s[:k]
        norm = np.sqrt(np.sum(s * s))
        return s / norm, Vh[:k], norm, w
