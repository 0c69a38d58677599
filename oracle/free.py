"""Free-particle references for the oracle (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

At U = 0, eq. (1) is quadratic: H = sum_{ab} h_ab b+_a b_b with the L x L
one-body matrix h (h_{j,j+1} = -J, h_{j,j+2} = -J_NNN, h_jj = K/2 (j-j_c)^2).
Heisenberg evolution gives b(t) = W b(0), W = exp(-i h t), so from a product
state with occupations occ_k

    <b+_a b_c>(t) = sum_k conj(W_ak) W_ck occ_k.

The same formula holds for free fermions from a Slater product state, and
hard-core bosons with nearest-neighbour hopping only map onto free fermions
with no Jordan-Wigner string on NN terms; so for n_max = 1, J_NNN = 0 the
densities and NN correlators of eq. (5), (8) follow it at any U (Sec. III D
treats the free and the infinitely repulsive chain as the same limit for these
observables).

A Trotterised gate exp(-i h_j tau) of a quadratic three-site term is a
one-body 3 x 3 rotation, so the Trotterised one-body propagator reproduces a
TEBD run exactly (no truncation, n_max >= N), independent of the MPS code.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.special


def one_body_h(L, J, Jnnn, K, jc) -> np.ndarray:
    """L x L one-body matrix of eq. (1) at U = 0 (1-based site j = row + 1)."""
    h = np.zeros((L, L))
    for p in range(L - 1):
        h[p, p + 1] = h[p + 1, p] = -J
    for p in range(L - 2):
        h[p, p + 2] = h[p + 2, p] = -Jnnn
    for p in range(L):
        h[p, p] = 0.5 * K * (p + 1 - jc) ** 2
    return h


def propagator(h: np.ndarray, t: float) -> np.ndarray:
    """W = exp(-i h t) (scipy expm)."""
    return scipy.linalg.expm(-1j * t * h)


def correlations(W: np.ndarray, occ) -> np.ndarray:
    """G_ac = <b+_a b_c> = sum_k conj(W_ak) W_ck occ_k."""
    occ = np.asarray(occ, dtype=np.float64)
    return (W.conj() * occ[None, :]) @ W.T


def observables(W, occ):
    """(n_j, C_j = <b+_j b_{j+1}>) from the one-body propagator."""
    G = correlations(W, occ)
    L = G.shape[0]
    return np.real(np.diag(G)).copy(), np.array([G[p, p + 1] for p in range(L - 1)])


def _triple_one_body(j, L, J, Jnnn, K, jc) -> np.ndarray:
    """3 x 3 one-body matrix of the three-site term of triple j (1-based).

    The split shares each NN bond among the triples containing it and each
    on-site trap term among the triples containing that site (reading S);
    the multiplicities are recomputed here from their definition.
    """
    def cb(k):  # triples containing bond (k, k+1)
        return int(k - 1 >= 1) + int(k <= L - 2)

    def cs(k):  # triples containing site k
        return sum(1 for m in (k - 2, k - 1, k) if 1 <= m <= L - 2)

    h = np.zeros((3, 3))
    h[0, 2] = h[2, 0] = -Jnnn
    for p in range(2):
        h[p, p + 1] = h[p + 1, p] = -J / cb(j + p)
    for p in range(3):
        k = j + p
        h[p, p] = 0.5 * K * (k - jc) ** 2 / cs(k)
    return h


def trotter_propagator(L, J, Jnnn, K, jc, dt, n_steps) -> np.ndarray:
    """One-body propagator of n_steps of A(dt/2) B(dt/2) C(dt) B(dt/2) A(dt/2).

    Layers by triple start j mod 3 (A: 1, B: 2, C: 0); within a layer the
    3 x 3 blocks act on disjoint sites.
    """
    def layer(res, tau):
        W = np.eye(L, dtype=np.complex128)
        for j in range(1, L - 1):
            if j % 3 == res:
                blk = scipy.linalg.expm(-1j * tau * _triple_one_body(j, L, J, Jnnn, K, jc))
                W[j - 1:j + 2, :] = blk @ W[j - 1:j + 2, :]
        return W

    A, B, C = layer(1, dt / 2), layer(2, dt / 2), layer(0, dt)
    step = A @ B @ C @ B @ A  # rightmost acts first
    return np.linalg.matrix_power(step, n_steps)


def _super_bond_one_body(k, Lp, J, Jnnn, K, jc) -> np.ndarray:
    """4 x 4 one-body matrix of super bond k (1-based) over physical sites 2k-1..2k+2 of a
    chain of Lp (even) sites, in the super-site split of Sec. II B: the NN hop (2k, 2k+1)
    and the NNN hops (2k-1, 2k+1), (2k, 2k+2) in full; the hop inside each super site and
    its trap terms divided by the number of super bonds holding that super site (1 or 2)."""
    L_eff = Lp // 2

    def share(kk):
        return sum(1 for b in (kk - 1, kk) if 1 <= b <= L_eff - 1)

    h = np.zeros((4, 4))
    h[1, 2] = h[2, 1] = -J
    h[0, 2] = h[2, 0] = h[1, 3] = h[3, 1] = -Jnnn
    for kk, (p0, p1) in ((k, (0, 1)), (k + 1, (2, 3))):
        c = share(kk)
        h[p0, p1] += -J / c
        h[p1, p0] += -J / c
        h[p0, p0] += 0.5 * K * (2 * kk - 1 - jc) ** 2 / c
        h[p1, p1] += 0.5 * K * (2 * kk - jc) ** 2 / c
    return h


def supersite_trotter_propagator(Lp, J, Jnnn, K, jc, dt, n_steps) -> np.ndarray:
    """One-body propagator (Lp x Lp, Lp even) of n_steps of the super-site split:
    odd super bonds for dt/2, even ones for dt, odd ones for dt/2."""
    L_eff = Lp // 2

    def layer(parity, tau):
        W = np.eye(Lp, dtype=np.complex128)
        for k in range(1, L_eff):
            if k % 2 == parity:
                blk = scipy.linalg.expm(-1j * tau * _super_bond_one_body(k, Lp, J, Jnnn, K, jc))
                W[2 * k - 2:2 * k + 2, :] = blk @ W[2 * k - 2:2 * k + 2, :]
        return W

    odd, even = layer(1, dt / 2), layer(0, dt)
    return np.linalg.matrix_power(odd @ even @ odd, n_steps)


def bessel_bulk(t, J=1.0):
    """Uniform NN chain, odd sites occupied, far from the edges (closed form).

    n_occ = (1 + J0(4Jt))/2, n_empty = (1 - J0(4Jt))/2 and the current from an
    occupied site into its right neighbour, 2J Im C_j = J J1(4Jt).
    From W_jk = i^{j-k} J_{j-k}(2Jt) and Neumann's addition theorem.
    """
    x = 4.0 * J * np.asarray(t, dtype=np.float64)
    j0 = scipy.special.jv(0, x)
    return 0.5 * (1 + j0), 0.5 * (1 - j0), J * scipy.special.jv(1, x)
