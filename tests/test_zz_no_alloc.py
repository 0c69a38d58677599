"""GPU test of tebd_bond_correlator_noalloc, the allocation-free correlator.

It serves callers that cannot allocate device memory when they need C_j
(a fixed memory budget, a framework allocator that owns all device memory,
or a loop where cudaMalloc would synchronise the device).  The test calls it
through the C ABI with caller-owned device buffers and checks:
  * both Re C_j and Im C_j of every bond of an evolved L = 8 state against the
    CPU oracle's correlators (eq. (5)), and 2 J Im C_j against the currents of
    tebd_measure, the existing entry point, on two calls in a row;
  * seeded random tensors at the scratch capacity (chi_l = chi_m = chi_r = 64,
    d = 8) and at a skewed shape (1, 64, 3, 8) against a numpy einsum of
    C = sum conj(theta[a,s,t,b]) <s t|b+ (x) b|s' t'> theta[a,s',t',b],
    theta = lam (.) B_left B_right.
This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _call(lib, Bl, laml, Br, stream):
    import torch
    chi_l, d, chi_m = Bl.shape
    chi_r = Br.shape[2]
    tBl = torch.from_numpy(np.ascontiguousarray(Bl, dtype=np.complex128).view(np.float64).ravel()).cuda()
    tBr = torch.from_numpy(np.ascontiguousarray(Br, dtype=np.complex128).view(np.float64).ravel()).cuda()
    tl = torch.from_numpy(np.ascontiguousarray(laml, dtype=np.float64)).cuda()
    tC = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    st = lib.tebd_bond_correlator_noalloc(
        ctypes.c_void_p(tBl.data_ptr()), ctypes.c_void_p(tl.data_ptr()), ctypes.c_void_p(tBr.data_ptr()),
        chi_l, chi_m, chi_r, d, ctypes.c_void_p(tC.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return complex(float(tC[0].item()), float(tC[1].item()))


def _run_bonds(lib, g, stream):
    out = []
    for k in range(g.L - 1):
        Bl, laml = g.get_site(k)
        Br, _ = g.get_site(k + 1)
        out.append(_call(lib, Bl, laml, Br, stream))
    return np.array(out)


def _einsum_correlator(Bl, laml, Br):
    d = Bl.shape[1]
    b = np.diag(np.sqrt(np.arange(1, d, dtype=np.float64)), 1)  # b|n> = sqrt(n)|n-1>
    theta = np.einsum("a,asm,mtb->astb", laml, Bl, Br)
    # <s t| b+ (x) b |s' t'> = (b+)_{s s'} b_{t t'}
    return np.einsum("astb,su,tv,auvb->", theta.conj(), b.T, b, theta)


def test_noalloc_correlator_matches_oracle_and_measure(lib):
    import torch
    from oracle.tebd import TEBD as OracleTEBD
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.PARITY_L8
    stream = torch.cuda.current_stream()
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, stream=stream.cuda_stream)
    g.init_product(wl.occupation())
    g.step(40)
    _, cur = g.measure()
    o = OracleTEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt)
    o.init_product(wl.occupation())
    o.step(40)
    C_o = o.correlators()
    assert np.max(np.abs(cur)) > 1e-3 and np.max(np.abs(C_o.real)) > 1e-3  # a non-trivial state
    first = _run_bonds(lib, g, stream)
    second = _run_bonds(lib, g, stream)
    for C in (first, second):
        assert np.max(np.abs(C.real - C_o.real)) < 1e-9
        assert np.max(np.abs(C.imag - C_o.imag)) < 1e-9
        assert np.max(np.abs(2.0 * wl.J * C.imag - cur)) < 1e-12
    g.close()


@pytest.mark.parametrize("shape", [(64, 64, 64, 8), (1, 64, 3, 8), (64, 1, 64, 2), (7, 33, 64, 5)])
def test_noalloc_correlator_random_tensors(lib, shape):
    import torch
    chi_l, chi_m, chi_r, d = shape
    rng = np.random.Generator(np.random.PCG64([workloads.SEED, *shape]))
    Bl = rng.standard_normal((chi_l, d, chi_m)) + 1j * rng.standard_normal((chi_l, d, chi_m))
    Br = rng.standard_normal((chi_m, d, chi_r)) + 1j * rng.standard_normal((chi_m, d, chi_r))
    lam = rng.uniform(0.1, 1.0, chi_l)
    ref = _einsum_correlator(Bl, lam, Br)
    stream = torch.cuda.current_stream()
    for _ in range(2):  # two calls in a row share the scratch
        C = _call(lib, Bl, lam, Br, stream)
        assert abs(C - ref) <= 1e-12 * max(1.0, abs(ref)), (shape, C, ref)


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.tebd_bond_correlator_noalloc(p, p, p, 65, 4, 4, 4, p, None) == -8
    assert lib.tebd_bond_correlator_noalloc(p, p, p, 4, 4, 4, 9, p, None) == -8
    assert lib.tebd_bond_correlator_noalloc(None, p, p, 4, 4, 4, 4, p, None) == -1
    assert lib.tebd_strerror(-8) == b"size exceeds the fixed scratch capacity"
