"""Exact diagonalisation pins for the TEBD oracle (dense, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Two independent references for small chains:

* ``sector_*``: eq. (1) assembled directly in the Fock basis of the fixed-N
  sector (N is conserved, Sec. II B), diagonalised once, and evolved exactly:
  psi(t) = V exp(-i E t) V^+ psi0.  Shares nothing with the three-site split.
* ``dense_trotter``: the same gate sequence as the TEBD applied to the full
  d^L state vector with no MPS and no truncation.  It isolates the MPS
  machinery (theta, SVD, rebuild, canonical-form observables) from the gates.

The hopping action below is written on occupation tuples with explicit
sqrt factors (b+_i b_k |..n_i..n_k..> = sqrt((n_i+1) n_k) |..n_i+1..n_k-1..>),
not with the local-operator matrices of ``model``.
"""
from __future__ import annotations

import itertools

import numpy as np


def sector_basis(L: int, n_max: int, N: int):
    """All occupation tuples of L sites with sum N and each n_j <= n_max."""
    basis = [c for c in itertools.product(range(n_max + 1), repeat=L) if sum(c) == N]
    return basis, {c: i for i, c in enumerate(basis)}


def full_basis(L: int, n_max: int):
    """All d^L occupation tuples in row-major (site 1 slowest) order."""
    basis = list(itertools.product(range(n_max + 1), repeat=L))
    return basis, {c: i for i, c in enumerate(basis)}


def _hop(conf, i, k, n_max):
    """b+_i b_k |conf> -> (amplitude, new_conf) or None (0-based sites, i != k)."""
    if conf[k] == 0 or conf[i] == n_max:
        return None
    amp = np.sqrt((conf[i] + 1) * conf[k])
    new = list(conf)
    new[i] += 1
    new[k] -= 1
    return amp, tuple(new)


def hamiltonian(basis, index, L, n_max, U, J, Jnnn, K, jc) -> np.ndarray:
    """Dense matrix of eq. (1) on the given basis (1-based site j = index + 1)."""
    D = len(basis)
    H = np.zeros((D, D), dtype=np.complex128)
    for a, conf in enumerate(basis):
        diag = 0.0
        for p, n in enumerate(conf):
            j = p + 1
            diag += 0.5 * U * n * (n - 1) + 0.5 * K * (j - jc) ** 2 * n
        H[a, a] += diag
        for p in range(L):
            for dist, amp0 in ((1, -J), (2, -Jnnn)):
                q = p + dist
                if q >= L or amp0 == 0.0:
                    continue
                for i, k in ((p, q), (q, p)):  # b+_p b_q and b+_q b_p
                    r = _hop(conf, i, k, n_max)
                    if r is None:
                        continue
                    amp, new = r
                    b = index.get(new)
                    if b is not None:
                        H[b, a] += amp0 * amp
    return H


def sector_observables(psi, basis, index, L, n_max):
    """n_j (eq. (8)) and C_j = <b+_j b_{j+1}> (eq. (5)) of a sector state vector."""
    occ = np.array(basis, dtype=np.float64)
    prob = np.abs(psi) ** 2
    n = prob @ occ
    C = np.zeros(L - 1, dtype=np.complex128)
    for a, conf in enumerate(basis):
        if psi[a] == 0:
            continue
        for p in range(L - 1):
            r = _hop(conf, p, p + 1, n_max)
            if r is None:
                continue
            amp, new = r
            b = index.get(new)
            if b is not None:
                C[p] += np.conj(psi[b]) * amp * psi[a]
    return n, C


class SectorED:
    """Exact evolution in the fixed-N sector: psi(t) = V exp(-iEt) V^+ psi0."""

    def __init__(self, L, n_max, occ, U, J, Jnnn, K, jc):
        occ = tuple(int(x) for x in occ)
        self.L, self.n_max = L, n_max
        self.basis, self.index = sector_basis(L, n_max, sum(occ))
        H = hamiltonian(self.basis, self.index, L, n_max, U, J, Jnnn, K, jc)
        self.E, self.V = np.linalg.eigh(H)
        psi0 = np.zeros(len(self.basis), dtype=np.complex128)
        psi0[self.index[occ]] = 1.0
        self.c0 = self.V.conj().T @ psi0

    def state(self, t):
        """psi(t) = V exp(-i E t) V^+ psi0 in the fixed-N sector (exact evolution under eq. (1))."""
        return self.V @ (np.exp(-1j * self.E * t) * self.c0)

    def observables(self, t):
        """(n_j, C_j) of eqs. (8), (5) at time t."""
        return sector_observables(self.state(t), self.basis, self.index, self.L, self.n_max)


# -- dense Trotterised evolution ---------------------------------------------------

def apply_three_site(psi: np.ndarray, G: np.ndarray, i: int, d: int) -> np.ndarray:
    """Apply a d^3 x d^3 gate to sites (i, i+1, i+2) (0-based) of psi[(d,)*L]."""
    L = psi.ndim
    x = np.moveaxis(psi, (i, i + 1, i + 2), (0, 1, 2)).reshape(d ** 3, -1)
    x = (G @ x).reshape((d, d, d) + tuple(np.delete(psi.shape, (i, i + 1, i + 2))))
    return np.moveaxis(x, (0, 1, 2), (i, i + 1, i + 2)).reshape((d,) * L)


def dense_product(occ, d):
    """Product state |occ_1 ... occ_L> (eq. (2) form) as a dense array of shape (d,)*L."""
    L = len(occ)
    psi = np.zeros((d,) * L, dtype=np.complex128)
    psi[tuple(int(x) for x in occ)] = 1.0
    return psi


def dense_trotter_step(psi, gate_of, schedule, d):
    """One step of the layer schedule on the dense vector; gate_of(j, tau) gives G_j."""
    for triples, tau in schedule:
        for j in triples:
            psi = apply_three_site(psi, gate_of(j, tau), j - 1, d)
    return psi


def dense_observables(psi: np.ndarray):
    """n_j and C_j = <b+_j b_{j+1}> of a dense state psi[(d,)*L] by index shifts."""
    L, d = psi.ndim, psi.shape[0]
    nvals = np.arange(d, dtype=np.float64)
    prob = np.abs(psi) ** 2
    n = np.empty(L)
    for j in range(L):
        n[j] = np.sum(np.moveaxis(prob, j, -1) @ nvals)
    C = np.empty(L - 1, dtype=np.complex128)
    sq = np.sqrt(np.arange(1, d, dtype=np.float64))  # sqrt(1..d-1)
    for j in range(L - 1):
        x = np.moveaxis(psi, (j, j + 1), (0, 1))
        # (b_{j+1} psi)[nj, m-1] = sqrt(m) psi[nj, m]; then b+_j raises nj-1 -> nj with sqrt(nj)
        # <psi| b+_j b_{j+1} |psi> = sum conj(psi[nj+1, m-1]) sqrt(nj+1) sqrt(m) psi[nj, m]
        lhs = x[1:, :-1]   # psi[nj+1, m-1]
        rhs = x[:-1, 1:]   # psi[nj, m]
        w = sq[:, None] * sq[None, :]  # sqrt(nj+1) * sqrt(m)
        C[j] = np.sum(np.conj(lhs) * (w.reshape(w.shape + (1,) * (x.ndim - 2)) * rhs))
    return n, C


def embed_three_site(h: np.ndarray, i: int, L: int, d: int) -> np.ndarray:
    """h acting on sites (i, i+1, i+2) as a d^L x d^L dense matrix (small L only)."""
    left = np.eye(d ** i)
    right = np.eye(d ** (L - i - 3))
    return np.kron(np.kron(left, h), right)
