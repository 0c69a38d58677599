"""CPU-side checks of the C-ABI library: it loads, exports every declared symbol,
and its host-only gate builder matches the oracle (no GPU compute)."""
import os
import re

import numpy as np
import pytest

from oracle import model
from paper_2401_05301_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_05301_gb300 import build
    build.build()
    return binding.load()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ptebd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tebd_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(binding.SIGNATURES)


def test_strerror(lib):
    assert lib.tebd_strerror(0) == b"ok"
    assert lib.tebd_strerror(-7) == b"non-finite singular values"


@pytest.mark.parametrize("n_max,L,j", [(1, 5, 1), (2, 6, 2), (3, 8, 3), (3, 8, 6), (4, 64, 30), (7, 6, 2)])
def test_host_gate_matches_oracle(lib, n_max, L, j):
    U, J, Jnnn, K, jc = 5.0, 1.0, 0.1, 0.003, (L + 1) / 2
    for tau in (0.005, 0.01):
        G = binding.gate_host(L, n_max, U, J, Jnnn, K, jc, j, tau)
        ref = model.gate(model.three_site_term(j, L, n_max, U, J, Jnnn, K, jc), tau)
        assert np.max(np.abs(G - ref)) < 1e-13
        assert np.max(np.abs(G.conj().T @ G - np.eye(len(G)))) < 1e-13


@pytest.mark.parametrize("sim,j", [("a", 1), ("d", 1), ("d", 60), ("d", 119)])
def test_host_gate_paper_setup(lib, sim, j):
    """The paper's setup (L = 121, d = 5, Table Ib, dt = 0.05 pi/2): at the chain ends the
    trap puts up to K/2 60^2 n = 209 on the diagonal of a three-site term, so these gates
    test the host eigen-solver far from the small-trap workloads."""
    import workloads
    wl = workloads.paper_run(sim, 27, 40)
    for tau in (wl.dt / 2, wl.dt):
        G = binding.gate_host(wl.L, wl.n_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, j, tau)
        ref = model.gate(model.three_site_term(j, wl.L, wl.n_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc), tau)
        assert np.max(np.abs(G - ref)) < 2e-13
        assert np.max(np.abs(G.conj().T @ G - np.eye(len(G)))) < 1e-13


def test_host_gate_rejects_bad_args(lib):
    out = np.empty(2 * 64 ** 2)
    ptr = out.ctypes.data_as(binding._P_double)
    assert lib.tebd_gate_host(2, 3, 1, 1, 0, 0, 1, 1, 0.1, ptr) == -1   # L < 3
    assert lib.tebd_gate_host(8, 3, 1, 1, 0, 0, 1, 7, 0.1, ptr) == -1   # j > L-2
    assert lib.tebd_gate_host(8, 3, float("nan"), 1, 0, 0, 1, 1, 0.1, ptr) == -1


def test_host_jacobi_sweep_limit_reports_not_converged(lib):
    """The host eigen-solver's sweep limit: one cyclic sweep cannot diagonalise a
    64 x 64 three-site term to 1e-32 of its norm, so the call reports
    TEBD_ERR_NOT_CONVERGED; with the default limit the same gate is built and
    equals tebd_gate_host."""
    L, n_max, U, J, Jnnn, K, jc, j, tau = 8, 3, 5.0, 1.0, 0.1, 0.003, 4.5, 3, 0.01
    with pytest.raises(binding.TEBDError) as e:
        binding.gate_host_sweeps(L, n_max, U, J, Jnnn, K, jc, j, tau, 1)
    assert e.value.status == -5
    G = binding.gate_host_sweeps(L, n_max, U, J, Jnnn, K, jc, j, tau, 60)
    assert np.array_equal(G, binding.gate_host(L, n_max, U, J, Jnnn, K, jc, j, tau))
    out = np.empty(2 * 64 ** 2)
    assert lib.tebd_gate_host_sweeps(L, n_max, U, J, Jnnn, K, jc, j, tau, 0,
                                     out.ctypes.data_as(binding._P_double)) == -1


@pytest.mark.parametrize("L,n_max", [(7, 1), (8, 2), (5, 3), (6, 4)])
def test_host_supersite_gate_matches_oracle(lib, L, n_max):
    """tebd_gate_host_supersite (block-wise exponential of the super bond term)
    against the super-site oracle's exp(-i h_k tau) of its own bond term, every bond."""
    from oracle import supersite
    U, J, Jnnn, K, jc, tau = 3.0, 1.0, 0.2, 0.05, (L + 1) / 2, 0.025
    L_eff = supersite.padded_length(L) // 2
    for k in range(1, L_eff):
        G = binding.gate_host_supersite(L, n_max, U, J, Jnnn, K, jc, k, tau)
        ref = model.gate(supersite.bond_term(k, L, n_max, U, J, Jnnn, K, jc), tau)
        assert np.max(np.abs(G - ref)) < 1e-13, k
        assert np.max(np.abs(G.conj().T @ G - np.eye(len(G)))) < 1e-13


def test_host_supersite_gate_paper_setup(lib):
    """L = 121 padded to 122 (61 super sites), d = 5, Table Ib set a: the end bonds carry
    the largest trap terms (|h| ~ 260, so |E tau| ~ 20 rad at tau = dt, and each side's
    phases carry rounding of order eps |E tau| over blocks of up to 85 states: bound 5e-13)."""
    import workloads
    from oracle import supersite
    wl = workloads.paper_run("a", 27, 40)
    for k in (1, 30, 60):
        G = binding.gate_host_supersite(wl.L, wl.n_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, k, wl.dt)
        ref = model.gate(supersite.bond_term(k, wl.L, wl.n_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc), wl.dt)
        assert np.max(np.abs(G - ref)) < 5e-13
        assert np.max(np.abs(G.conj().T @ G - np.eye(len(G)))) < 1e-13


def test_host_supersite_gate_rejects_bad_args(lib):
    out = np.empty(2 * 5 ** 8)
    ptr = out.ctypes.data_as(binding._P_double)
    assert lib.tebd_gate_host_supersite(2, 1, 1, 1, 0, 0, 1, 1, 0.1, ptr) == -1   # L < 3
    assert lib.tebd_gate_host_supersite(8, 1, 1, 1, 0, 0, 1, 4, 0.1, ptr) == -1   # k > L_eff - 1
    assert lib.tebd_gate_host_supersite(8, 5, 1, 1, 0, 0, 1, 1, 0.1, ptr) == -1   # n_max > 4
    assert lib.tebd_gate_host_supersite(8, 2, 1, float("inf"), 0, 0, 1, 1, 0.1, ptr) == -1
