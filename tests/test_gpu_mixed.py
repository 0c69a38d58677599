"""Mixed precision: the 3xTF32 tensor-core contractions.

(1) tebd_zgemm through the C ABI against a numpy FP64 product on ragged,
multi-tile shapes (both op(B) forms): relative error ~5e-7 of |A||B|.
(2) Whole runs with precision = 1 against the FP64 oracle: the stated bound
for the mixed path is 1e-5 on densities and currents; the measured maximum
is printed for every run.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle.tebd import TEBD as OracleTEBD

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-5


def _zgemm(lib, precision, opB, A, B, alpha=1.0):
    import torch
    M, K = A.shape
    N = B.shape[1] if opB == 0 else B.shape[0]
    tA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    tB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    tC = torch.full((M, N), complex("nan"), dtype=torch.complex128, device="cuda")
    st = lib.tebd_zgemm(precision, opB, M, N, K, alpha, ctypes.c_void_p(tA.data_ptr()), K,
                        ctypes.c_void_p(tB.data_ptr()), B.shape[1], ctypes.c_void_p(tC.data_ptr()), N,
                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return tC.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (37, 5, 3), (128, 128, 16), (300, 200, 70), (129, 257, 33),
                                   (64, 600, 125)])
@pytest.mark.parametrize("opB", [0, 1])
def test_zgemm_tf32x3_matches_fp64(lib, M, N, K, opB):
    rng = np.random.default_rng(M * 1000 + N * 10 + K + opB)
    A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    B = rng.standard_normal((K, N) if opB == 0 else (N, K)) + 1j * rng.standard_normal((K, N) if opB == 0 else (N, K))
    ref = 0.7 * (A @ (B if opB == 0 else B.conj().T))
    scale = (np.abs(A) @ np.abs(B if opB == 0 else B.T)) * 0.7
    c64 = _zgemm(lib, 0, opB, A, B, 0.7)
    c32 = _zgemm(lib, 1, opB, A, B, 0.7)
    assert np.max(np.abs(c64 - ref) / scale) < 1e-14
    err = np.max(np.abs(c32 - ref) / scale)
    assert err < 1e-6, err


@pytest.mark.parametrize("K", [256, 1024, 4096])
def test_zgemm_tf32x3_no_accumulation_bias(lib, K):
    """Same-sign data over a long K: the tensor core's round-towards-zero FP32
    accumulation must not build up (each 32-real slab is drained into FP32
    registers with round-to-nearest adds): the mean error stays ~0 and the
    maximum grows only like sqrt(K) (unbiased FP32 sums)."""
    rng = np.random.default_rng(K)
    A = rng.uniform(0, 1, (256, K)) + 1j * rng.uniform(0, 1, (256, K))
    B = rng.uniform(0, 1, (K, 192)) + 1j * rng.uniform(0, 1, (K, 192))
    ref = A @ B
    c32 = _zgemm(lib, 1, 0, A, B)
    scale = np.abs(A) @ np.abs(B)
    err = (c32 - ref) / scale
    print(f"K={K}: max rel {np.max(np.abs(err)):.2e}, mean {np.mean(err.real):+.2e}")
    assert np.max(np.abs(err)) < 3e-6
    assert abs(np.mean(err.real)) < 1e-7


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (37, 5, 3), (128, 32, 16), (300, 200, 70), (129, 257, 300),
                                   (64, 600, 125), (256, 96, 1030)])
@pytest.mark.parametrize("opB", [0, 1])
def test_zgemm_exact_digits_matches_fp64(lib, M, N, K, opB):
    """precision 2 (exact-digit products on the bf16 tensor cores) against numpy
    FP64: rows spanning 30 orders of magnitude, error below 2e-15 of |A||B|
    (the FP64 path's own bound here is 1e-14)."""
    rng = np.random.default_rng(7 * M + 3 * N + K + opB)
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * 10.0 ** rng.uniform(-15, 15, (M, 1))
    Bs = (K, N) if opB == 0 else (N, K)
    B = (rng.standard_normal(Bs) + 1j * rng.standard_normal(Bs)) * 10.0 ** rng.uniform(-8, 8, (Bs[0], 1))
    opb = B if opB == 0 else B.conj().T
    ref = 1.3 * (A @ opb)
    scale = 1.3 * (np.abs(A) @ np.abs(opb))
    c2 = _zgemm(lib, 2, opB, A, B, 1.3)
    err = np.max(np.abs(c2 - ref) / scale)
    print(f"exact-digit zgemm {M}x{N}x{K} opB={opB}: max error / (|A||B|) = {err:.2e}")
    assert err < 2e-15, err


def test_zgemm_exact_digits_gram_is_hermitian(lib):
    """A A^+ through precision 2: Hermitian to the last bit on the diagonal's
    imaginary part (digits of -x are the negated digits of x)."""
    rng = np.random.default_rng(11)
    A = rng.standard_normal((200, 333)) + 1j * rng.standard_normal((200, 333))
    H = _zgemm(lib, 2, 1, A, A)
    assert np.all(np.diag(H).imag == 0.0)
    ref = A @ A.conj().T
    assert np.max(np.abs(H - ref)) / np.max(np.abs(ref)) < 1e-15


def _compare_mixed(lib, wl, n_steps, every):
    from paper_2401_05301_gb300 import TEBD
    args = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
                dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    g = TEBD(**args, precision=1)
    o = OracleTEBD(**args)
    occ = wl.occupation()
    g.init_product(occ)
    o.init_product(occ)
    dn = dc = 0.0
    for _ in range(every, n_steps + 1, every):
        g.step(every)
        o.step(every)
        n_g, cur_g = g.measure()
        dn = max(dn, np.max(np.abs(n_g - o.densities())))
        dc = max(dc, np.max(np.abs(cur_g - o.currents())))
    g.close()
    return dn, dc


def test_mixed_L8_against_fp64_oracle(lib):
    dn, dc = _compare_mixed(lib, workloads.PARITY_L8, 200, 20)
    print(f"mixed L8 (t=2): max |dn| = {dn:.2e}, max |dcurrent| = {dc:.2e}")
    assert dn < MIXED_TOL and dc < MIXED_TOL


def test_mixed_L32_against_fp64_oracle(lib):
    dn, dc = _compare_mixed(lib, workloads.TRUNC_L32, 60, 20)
    print(f"mixed L32 (t=0.6): max |dn| = {dn:.2e}, max |dcurrent| = {dc:.2e}")
    assert dn < MIXED_TOL and dc < MIXED_TOL
