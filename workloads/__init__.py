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


def random_product_states(L: int, n_max: int, count: int, seed: int = SEED):
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    return [rng.integers(0, n_max + 1, size=L) for _ in range(count)]
