"""Hamiltonian of eq. (1) and its exact three-site gates (oracle; FP64, numpy).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The model (paper Sec. I A, eq. (1)) is the open Bose-Hubbard chain j = 1..L

    H = U/2 sum_j n_j (n_j - 1)  -  J sum_{j<L} (b+_j b_{j+1} + h.c.)
        + K/2 sum_j (j - j_c)^2 n_j  -  J_NNN sum_{j<L-1} (b+_j b_{j+2} + h.c.)

with the boson truncated at n_max quanta per site (Sec. II B: d = n_max + 1).

Reading S (the paper groups sites into super sites instead, Sec. II B; the
three-site split is this library's choice for the NNN term): H is written as
sum_{j=1}^{L-2} h_j, where h_j acts on the triple (j, j+1, j+2) and holds

  * the NNN hop of that triple, with weight 1,
  * each NN hop (k, k+1) inside the triple divided by c_b(k), the number of
    triples that contain bond k,
  * each on-site term of a site k in the triple divided by c_s(k), the number
    of triples that contain site k,

so that sum_j h_j equals eq. (1) exactly (checked in the tests by building eq.
(1) independently in the Fock basis).
"""
from __future__ import annotations

import numpy as np


def local_ops(n_max: int):
    """Annihilator b, number operator n and identity on C^d, d = n_max + 1.

    b|n> = sqrt(n)|n-1>, truncated Fock space of Sec. II B (n_max).
    """
    d = n_max + 1
    b = np.zeros((d, d), dtype=np.complex128)
    for n in range(1, d):
        b[n - 1, n] = np.sqrt(n)
    num = np.diag(np.arange(d, dtype=np.float64)).astype(np.complex128)
    return b, num, np.eye(d, dtype=np.complex128)


def bond_multiplicity(k: int, L: int) -> int:
    """c_b(k): number of triples (j, j+1, j+2), 1 <= j <= L-2, containing bond (k, k+1).

    Reading S.  Bond k (1-based, 1 <= k <= L-1) lies in triple j iff j <= k <= j+1.
    """
    return sum(1 for j in (k - 1, k) if 1 <= j <= L - 2)


def site_multiplicity(k: int, L: int) -> int:
    """c_s(k): number of triples containing site k (1-based).  Reading S."""
    return sum(1 for j in (k - 2, k - 1, k) if 1 <= j <= L - 2)


def three_site_term(j: int, L: int, n_max: int, U: float, J: float, Jnnn: float,
                    K: float, jc: float) -> np.ndarray:
    """h_j on the triple (j, j+1, j+2), 1-based j in [1, L-2]; a d^3 x d^3 matrix.

    Basis order s1 (x) s2 (x) s3 with s3 fastest.  Terms of eq. (1) shared out
    among the triples as in reading S.
    """
    if L < 3 or not (1 <= j <= L - 2):
        raise ValueError("three-site terms need L >= 3 and 1 <= j <= L-2")
    b, num, one = local_ops(n_max)
    bd = b.conj().T

    def on(op, pos):  # embed a one-site operator at position pos in {0,1,2}
        mats = [one, one, one]
        mats[pos] = op
        return np.kron(np.kron(mats[0], mats[1]), mats[2])

    def hop(p, q):  # b+_p b_q + h.c. on positions p != q
        mats = [one, one, one]
        mats[p] = bd
        mats[q] = b
        t = np.kron(np.kron(mats[0], mats[1]), mats[2])
        return t + t.conj().T

    h = -Jnnn * hop(0, 2)
    for p in range(2):  # NN bonds (j+p, j+p+1)
        k = j + p
        h = h + (-J / bond_multiplicity(k, L)) * hop(p, p + 1)
    for p in range(3):
        k = j + p
        onsite = 0.5 * U * (num @ (num - one)) + 0.5 * K * (k - jc) ** 2 * num
        h = h + on(onsite, p) / site_multiplicity(k, L)
    return h


def gate(h: np.ndarray, tau: float) -> np.ndarray:
    """Exact exponential G = exp(-i h tau) of a Hermitian local term.

    Second-order Trotter gates (Sec. II B, Appendix A) are exact exponentials
    of the local terms; computed as V diag(exp(-i E tau)) V^+ from eigh.
    """
    E, V = np.linalg.eigh(h)
    return (V * np.exp(-1j * E * tau)) @ V.conj().T


def layer_of(j: int) -> str:
    """Layer label of triple j (1-based): A if j = 1 mod 3, B if 2, C if 0.

    Triples whose starting sites agree mod 3 are disjoint, so each layer is a
    set of independent local updates (the data-parallel bulk).
    """
    return {1: "A", 2: "B", 0: "C"}[j % 3]


def step_schedule(L: int, dt: float, order: int = 2):
    """One step of the layer schedule: a list of (list_of_triples_1based, tau).

    order 2: the symmetric step A(dt/2) B(dt/2) C(dt) B(dt/2) A(dt/2) (Strang
    splitting of the three layer Hamiltonians; second-order Trotter, Sec. II B /
    Appendix A).  order 4: Suzuki's fourth-order fractal composition of that step,
    S2(p dt) S2(p dt) S2((1-4p) dt) S2(p dt) S2(p dt) with p = 1/(4 - 4^(1/3)); the
    paper cross-checks its second-order results against a fourth-order split
    (Appendix A), without fixing the composition.  Reading M: adjacent half-step
    layers (inside a step or across steps) are never merged.
    """
    trip = {lab: [j for j in range(1, L - 1) if layer_of(j) == lab] for lab in "ABC"}

    def s2(tau):
        return [(trip["A"], tau / 2), (trip["B"], tau / 2), (trip["C"], tau),
                (trip["B"], tau / 2), (trip["A"], tau / 2)]

    if order == 2:
        return s2(dt)
    if order == 4:
        p = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
        q = 1.0 - 4.0 * p
        return s2(p * dt) + s2(p * dt) + s2(q * dt) + s2(p * dt) + s2(p * dt)
    raise ValueError("order must be 2 or 4")


def cdw_occupation(L: int) -> np.ndarray:
    """|1,0,1,0,...> on j = 1..L (occupied odd sites, reading I)."""
    return np.array([1 if (j % 2 == 1) else 0 for j in range(1, L + 1)], dtype=np.int64)
