"""GPU test of tebd_bond_correlator_noalloc, the allocation-free correlator.

It serves callers that cannot allocate device memory when they need C_j
(a fixed memory budget, a framework allocator that owns all device memory,
or a loop where cudaMalloc would synchronise the device).  The test calls it
through the C ABI with caller-owned device buffers and checks 2 J Im C_j
against the currents of tebd_measure, the existing entry point, on two
calls in a row.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _run_bonds(lib, g, stream, J):
    import torch
    L = g.L
    out = []
    for k in range(L - 1):
        Bl, laml = g.get_site(k)
        Br, _ = g.get_site(k + 1)
        chi_l, d, chi_m = Bl.shape
        chi_r = Br.shape[2]
        tBl = torch.from_numpy(np.ascontiguousarray(Bl).view(np.float64).ravel()).cuda()
        tBr = torch.from_numpy(np.ascontiguousarray(Br).view(np.float64).ravel()).cuda()
        tl = torch.from_numpy(np.ascontiguousarray(laml)).cuda()
        tC = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = lib.tebd_bond_correlator_noalloc(
            ctypes.c_void_p(tBl.data_ptr()), ctypes.c_void_p(tl.data_ptr()), ctypes.c_void_p(tBr.data_ptr()),
            chi_l, chi_m, chi_r, d, ctypes.c_void_p(tC.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0, st
        torch.cuda.synchronize()
        out.append(2.0 * J * float(tC[1].item()))
    return np.array(out)


def test_noalloc_correlator_matches_measure(lib):
    import torch
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.PARITY_L8
    stream = torch.cuda.current_stream()
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, stream=stream.cuda_stream)
    g.init_product(wl.occupation())
    g.step(40)
    _, cur = g.measure()
    assert np.max(np.abs(cur)) > 1e-3  # a non-trivial state
    first = _run_bonds(lib, g, stream, wl.J)
    second = _run_bonds(lib, g, stream, wl.J)
    assert np.max(np.abs(first - cur)) < 1e-12
    assert np.max(np.abs(second - cur)) < 1e-12
    g.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    import torch
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    assert lib.tebd_bond_correlator_noalloc(p, p, p, 65, 4, 4, 4, p, None) == -8
    assert lib.tebd_bond_correlator_noalloc(p, p, p, 4, 4, 4, 9, p, None) == -8
    assert lib.tebd_bond_correlator_noalloc(None, p, p, 4, 4, 4, 4, p, None) == -1
    assert lib.tebd_strerror(-8) == b"size exceeds the fixed scratch capacity"
