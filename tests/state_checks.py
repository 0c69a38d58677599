"""Properties of a B-form state that hold at any size (used where the oracle cannot
redo an update in seconds): right-canonical site tensors, normalised bond vectors,
and the particle number carried by the canonical-form densities.

Right-canonicality is exact only while nothing is truncated: the division-free
update B_i = C V1^+ / ||s|| gives B_i B_i^+ = C P C^+ / ||s||^2 with P the projector
onto the kept singular vectors, which leaves the identity by about the discarded
weight over the smallest kept lambda^2 (2e-5 on an L = 8 run with eps = 1e-12).
The bond vectors stay normalised exactly, and the particle number moves at
O(w_total)."""
import numpy as np


def canonical_error(B) -> float:
    """max over sites of |B_k B_k^+ - I| with B_k viewed as chi_k x (d chi_{k+1})."""
    worst = 0.0
    for b in B:
        M = np.asarray(b).reshape(b.shape[0], -1)
        worst = max(worst, float(np.max(np.abs(M @ M.conj().T - np.eye(M.shape[0])))))
    return worst


def norm_error(lam) -> float:
    """max over bonds of |sum_a lam_a^2 - 1|."""
    return max(abs(float(np.sum(np.asarray(x) ** 2)) - 1.0) for x in lam)


def particle_number(B, lam) -> float:
    """sum_j n_j from the canonical form, n_j = sum lam_{j,a}^2 |B_j[a, s, b]|^2 s (eq. (8))."""
    total = 0.0
    for k, b in enumerate(B):
        s = np.arange(b.shape[1], dtype=np.float64)
        w = (np.asarray(lam[k]) ** 2)[:, None, None] * np.abs(b) ** 2
        total += float(np.sum(w.sum(axis=(0, 2)) * s))
    return total
