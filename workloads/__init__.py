"""Seeded synthetic inputs shared by the tests, the bench and the CPU oracle arm.

This module holds workload definitions and random-number draws only: no part
of the TEBD method's arithmetic lives here, and it imports neither the oracle
nor the CUDA library.

Workloads (all CDW product states |1,0,1,0,...> on j = 1..L unless noted,
hbar = J = 1 units):

* ``PARITY_L8``   L=8, n_max=3 (d=4), N=4, U=5, J=1, J_NNN=0.1, K=0, dt=0.01,
                  t_end=4, chi_max=256 (no truncation), measure every 0.1.
* ``TRUNC_L32``   L=32, d=4, N=16, U=5, J_NNN=0.12, K=0.005, j_c=16.5,
                  dt=0.01, t_end=6, chi_max=256, discarded-weight cut 1e-10.
* ``MIXED_L64``   L=64, n_max=4 (d=5), N=32, U=3, J_NNN=0.1, K=0.003,
                  j_c=32.5, dt=0.005, t_end=8, chi_max=1024.
* ``BATCH48``     48 simulations with seeded L, U, J_NNN, K, chi_max draws.
* ``SERVE500``    500-request seeded Poisson stream (90% MIXED_L64-style,
                  10% L=100, d=4, chi_max=2048 jobs).
* ``paper_run``   the paper's own setup: L=121, d=5, flanked CDW of N bosons,
                  Table Ib parameters, dt = 0.05 pi/2, cuts 1e-12.

``synthetic_state`` builds the reproducible saturated state used to time the
update "at chi_max": chi_j = min(chi_max, d^min(j, L-j)), right-canonical B
from the QR of seeded complex Gaussian matrices, and lambda_j with
p_k proportional to exp(-8 k / chi_j).
``synthetic_state_u1`` is the same kind of state with U(1) charge labels
(block-structured B, labels = boson count left of each bond), for a path that
exploits particle-number conservation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED = 240105301


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    n_max: int
    chi_max: int
    U: float
    J: float
    Jnnn: float
    K: float
    jc: float
    dt: float
    t_end: float
    w_cut: float = 0.0
    eps_rel: float = 1e-12
    measure_every: int = 10
    occ: tuple = field(default=())

    @property
    def d(self) -> int:
        return self.n_max + 1

    def occupation(self) -> np.ndarray:
        if self.occ:
            return np.array(self.occ, dtype=np.int64)
        return cdw(self.L)

    @property
    def n_steps(self) -> int:
        return int(round(self.t_end / self.dt))


def cdw(L: int) -> np.ndarray:
    """|1,0,1,0,...>: occupied odd sites j = 1, 3, 5, ... (1-based)."""
    return np.array([1 if j % 2 == 1 else 0 for j in range(1, L + 1)], dtype=np.int64)


PARITY_L8 = Workload("parity_L8_d4_chi256", L=8, n_max=3, chi_max=256, U=5.0, J=1.0, Jnnn=0.1, K=0.0,
                     jc=4.5, dt=0.01, t_end=4.0, w_cut=0.0)
TRUNC_L32 = Workload("trunc_L32_d4_chi256", L=32, n_max=3, chi_max=256, U=5.0, J=1.0, Jnnn=0.12, K=0.005,
                     jc=16.5, dt=0.01, t_end=6.0, w_cut=1e-10)
MIXED_L64 = Workload("mixed_L64_d5_chi1024", L=64, n_max=4, chi_max=1024, U=3.0, J=1.0, Jnnn=0.1, K=0.003,
                     jc=32.5, dt=0.005, t_end=8.0, w_cut=0.0)
# The same physics on a 16-site chain: bonds 5..11 saturate at chi_max = 1024 (5^5 > 1024), so one
# step holds the chi_max = 1024, d = 5 local updates in about a minute of GPU time.
SAMPLE_L16_D5 = Workload("sample_L16_d5_chi1024", L=16, n_max=4, chi_max=1024, U=3.0, J=1.0, Jnnn=0.1, K=0.003,
                         jc=8.5, dt=0.005, t_end=8.0, w_cut=0.0)


def flanked_cdw(L: int, N: int) -> np.ndarray:
    """Sec. II C's initial state: a CDW of N bosons in the middle of the chain with empty flanks.

    The central site (1-based (L+1)/2, the paper's j = 0) is occupied, and so is every
    second site out to N occupied sites; every site at odd distance from the centre and
    both flanks are empty.  Needs L odd, N odd and 2N - 1 <= L.
    """
    if L % 2 == 0 or N % 2 == 0 or not (1 <= N and 2 * N - 1 <= L):
        raise ValueError("flanked CDW needs L odd, N odd and 2N - 1 <= L")
    c = (L - 1) // 2  # 0-based centre
    occ = np.zeros(L, dtype=np.int64)
    half = (N - 1) // 2
    occ[c - 2 * half:c + 2 * half + 1:2] = 1
    return occ


# Table Ib's four parameter sets (U, J_NNN, K; J = 1), J_NNN passed into eq. (1) as printed.
PAPER_PARAMS = {"a": (2.442, -0.12, 0.010), "b": (3.604, -0.08, 0.013),
                "c": (5.167, -0.05, 0.017), "d": (9.910, -0.03, 0.029)}


def paper_run(sim: str, N: int, chi_max: int, L: int = 121, n_steps: int = 100) -> Workload:
    """A run as the paper sets it up (Sec. II C): L = 121 sites, trap centred on the middle
    site, flanked CDW of N bosons, n_max = 4, dt = 0.05 pi/2, 100 steps, discarded-weight and
    relative cuts 1e-12, measured after every step.  The paper's chi_max values are 40, 200,
    1000 and 5000; its ensemble over N needs weights that exist only in a missing figure."""
    U, Jnnn, K = PAPER_PARAMS[sim]
    dt = 0.05 * np.pi / 2
    return Workload(f"paper_{sim}_L{L}_N{N}_chi{chi_max}", L=L, n_max=4, chi_max=chi_max, U=U, J=1.0,
                    Jnnn=Jnnn, K=K, jc=(L + 1) / 2, dt=dt, t_end=n_steps * dt, w_cut=1e-12,
                    eps_rel=1e-12, measure_every=1, occ=tuple(int(x) for x in flanked_cdw(L, N)))


def batch48(seed: int = SEED):
    """48 simulations: per simulation in order L, U, J_NNN, K, chi_max draws; d=4, dt=0.01, t_end=4."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for s in range(48):
        L = int(rng.choice(np.arange(16, 65, 8)))
        U = float(rng.uniform(2.0, 6.0))
        Jnnn = float(rng.uniform(0.0, 0.15))
        K = float(rng.uniform(0.0, 0.01))
        chi = int(rng.choice([64, 128, 256, 512]))
        out.append(Workload(f"batch{s}", L=L, n_max=3, chi_max=chi, U=U, J=1.0, Jnnn=Jnnn, K=K,
                            jc=(L + 1) / 2, dt=0.01, t_end=4.0))
    return out


def synthetic_bond_dims(L: int, d: int, chi_max: int):
    """chi_k for bonds k = 0..L (chi_0 = chi_L = 1): min(chi_max, d^min(k, L-k))."""
    out = []
    for k in range(L + 1):
        e = min(k, L - k)
        out.append(int(min(chi_max, d ** e)) if e < 40 else chi_max)
    return out


def synthetic_state(L: int, d: int, chi_max: int, seed: int = SEED, decay: float = 8.0):
    """Seeded saturated B-form state: (B list, lambda list, chi list).

    B_k has shape (chi_k, d, chi_{k+1}) with orthonormal rows when reshaped to
    chi_k x (d chi_{k+1}) (right-canonical); lambda_k has p_i ~ exp(-decay i / chi_k),
    normalised so that sum lambda^2 = 1.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    chi = synthetic_bond_dims(L, d, chi_max)
    B = []
    for k in range(L):
        a, b = chi[k], chi[k + 1]
        X = rng.standard_normal((d * b, a)) + 1j * rng.standard_normal((d * b, a))
        Q, _ = np.linalg.qr(X)  # (d b) x a with orthonormal columns
        B.append(np.ascontiguousarray(Q.conj().T).reshape(a, d, b))
    lam = []
    for k in range(L + 1):
        n = chi[k]
        p = np.exp(-decay * np.arange(n) / max(n, 1))
        lam.append(np.sqrt(p / p.sum()))
    return B, lam, chi


def _sector_counts(sites: int, n_max: int, N: int) -> np.ndarray:
    """Number of occupation strings of `sites` sites (0..n_max each) with each total 0..N."""
    c = np.zeros(N + 1, dtype=np.float64)
    c[0] = 1.0
    for _ in range(sites):
        nxt = np.zeros_like(c)
        for s in range(n_max + 1):
            nxt[s:] += c[:N + 1 - s]
        c = nxt
    return c


def synthetic_state_u1(L: int, d: int, chi_max: int, N: int, seed: int = SEED, decay: float = 8.0):
    """Seeded saturated B-form state with U(1) charge labels: (B, lambda, q).

    q[k] holds, for each Schmidt index of bond k, the boson count on the sites left of
    the bond (sorted ascending, so each charge is one contiguous run); B_k[a, s, b] is
    non-zero only where q[k+1][b] = q[k][a] + s, and each charge block of B_k has
    orthonormal rows (right-canonical), from the QR of a seeded complex Gaussian block.
    A charge c on bond k gets a share of chi_k = min(chi_max, d^min(k, L-k)) in
    proportion to its largest possible Schmidt rank, capped so that the rows of every
    block of B_k fit its columns.  lambda_k has p_i ~ exp(-decay i / chi_k), the largest
    values on the charges nearest the mean filling N k / L.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_max = d - 1
    if not (0 <= N <= L * n_max):
        raise ValueError("N out of range")
    chi = synthetic_bond_dims(L, d, chi_max)
    sizes = [None] * (L + 1)
    sizes[L] = {N: 1}
    for k in range(L - 1, 0, -1):  # right to left, so the column counts of bond k+1 are known
        left, right = _sector_counts(k, n_max, N), _sector_counts(L - k, n_max, N)
        rank = {c: min(left[c], right[N - c]) for c in range(N + 1) if left[c] > 0 and right[N - c] > 0}
        cols = {c: sum(sizes[k + 1].get(c + t, 0) for t in range(d)) for c in rank}
        cap = {c: int(min(rank[c], cols[c])) for c in rank if min(rank[c], cols[c]) >= 1}
        total = min(chi[k], sum(cap.values()))
        weight = np.array([float(cap[c]) for c in sorted(cap)])
        share = np.minimum(np.floor(total * weight / weight.sum()).astype(int), [cap[c] for c in sorted(cap)])
        share = np.maximum(share, 0)
        order = sorted(cap, key=lambda c: abs(c - N * k / L))
        i = 0
        while share.sum() < total:  # hand out the remainder, central charges first
            c = order[i % len(order)]
            j = sorted(cap).index(c)
            if share[j] < cap[c]:
                share[j] += 1
            i += 1
        sizes[k] = {c: int(n) for c, n in zip(sorted(cap), share) if n > 0}
    sizes[0] = {0: 1}
    q = [np.repeat(np.array(sorted(sz), dtype=np.int64), [sz[c] for c in sorted(sz)]) for sz in sizes]
    B = []
    for k in range(L):
        a_n, b_n = len(q[k]), len(q[k + 1])
        t = np.zeros((a_n, d, b_n), dtype=np.complex128)
        for c in sizes[k]:
            rows = np.flatnonzero(q[k] == c)
            cols = [(s, b) for s in range(d) for b in np.flatnonzero(q[k + 1] == c + s)]
            X = rng.standard_normal((len(cols), len(rows))) + 1j * rng.standard_normal((len(cols), len(rows)))
            Q, _ = np.linalg.qr(X)
            for ci, (s, b) in enumerate(cols):
                t[rows, s, b] = Q[ci].conj()
        B.append(t)
    lam = []
    for k in range(L + 1):
        n = len(q[k])
        p = np.exp(-decay * np.arange(n) / max(n, 1))
        rank_order = np.argsort(np.abs(q[k] - N * k / L), kind="stable")
        v = np.empty(n)
        v[rank_order] = np.sqrt(p / p.sum())
        lam.append(v)
    return B, lam, q


def gaussian_test_matrix(n: int, l: int, call: int, seed: int = SEED) -> np.ndarray:
    """The n x l complex Gaussian test matrix of the call-th randomized decomposition:
    drawn from its own stream, keyed by (seed, call), so every decomposition's draws are
    fixed whatever ran before it."""
    rng = np.random.Generator(np.random.PCG64([seed, 7, int(call)]))
    return rng.standard_normal((n, l)) + 1j * rng.standard_normal((n, l))


def random_product_states(L: int, n_max: int, count: int, seed: int = SEED):
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    return [rng.integers(0, n_max + 1, size=L) for _ in range(count)]
