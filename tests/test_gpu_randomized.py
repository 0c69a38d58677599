"""GPU randomized truncation (option "randomized": the randomized range finder of Sec. V's
reduced-rank randomized SVD, Halko-Martinsson-Tropp) against the randomized oracle
(oracle/randomized.py) given the same Gaussian test matrices.

Both sides receive the test matrix of every decomposition from workloads.gaussian_test_matrix,
keyed by the decomposition's index (layer by layer, triples in site order, cut 1 then cut 2),
so the same sketches are taken.  Compared: densities and currents (1e-9 for the FP64 and
exact-digit paths, 1e-5 mixed) and the kept bond dimension chi' of every bond.
"""
import numpy as np
import pytest

import workloads
from oracle.randomized import RandomizedTEBD

pytestmark = pytest.mark.gpu


def _omega(call, n, l):
    return workloads.gaussian_test_matrix(n, l, call)


def _run(wl, n_steps, every, precision=0, tol=1e-9, chi_max=None, **kw):
    from paper_2401_05301_gb300 import TEBD
    args = dict(L=wl.L, n_max=wl.n_max, chi_max=chi_max or wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K,
                jc=wl.jc, dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    g = TEBD(**args, precision=precision)
    g.set_option("randomized", 1)
    g.set_test_matrices(_omega)
    o = RandomizedTEBD(**args, omega_fn=lambda n, l, call: _omega(call, n, l), **kw)
    occ = wl.occupation()
    g.init_product(occ)
    o.init_product(occ)
    worst = 0.0
    for _ in range(every, n_steps + 1, every):
        g.step(every)
        o.step(every)
        n_g, cur_g = g.measure()
        err = max(np.max(np.abs(n_g - o.densities())), np.max(np.abs(cur_g - o.currents())))
        chi_g, chi_o = list(g.bond_dims()), o.chi()
        assert chi_g == chi_o or o.min_cut_gap < 1e-6, (chi_g, chi_o)
        assert err < tol, err
        worst = max(worst, err)
    g.close()
    return worst


@pytest.mark.parametrize("precision", [0, 2])
def test_randomized_L8_no_cut(lib, precision):
    """chi_max = 256 >= every Schmidt rank: the sketch holds the whole range."""
    worst = _run(workloads.PARITY_L8, 60, 20, precision)
    print(f"randomized L8 (precision {precision}): max |delta| = {worst:.2e}")


def test_randomized_L8_with_chi_cut(lib):
    """chi_max = 16 cuts the middle bonds: the oversampled sketch (l = 26) and two power
    iterations find the same leading values as the oracle's sketch."""
    worst = _run(workloads.PARITY_L8, 60, 20, 0, chi_max=16)
    print(f"randomized L8 chi_max=16: max |delta| = {worst:.2e}")


def test_randomized_L32_truncating(lib):
    worst = _run(workloads.TRUNC_L32, 30, 10, 0)
    print(f"randomized L32 (w_cut 1e-10): max |delta| = {worst:.2e}")


def test_randomized_mixed(lib):
    worst = _run(workloads.PARITY_L8, 60, 20, 1, tol=1e-5)
    print(f"randomized L8 mixed: max |delta| = {worst:.2e}")


def test_randomized_needs_a_source_and_refuses_blocks(lib):
    from paper_2401_05301_gb300 import TEBD, TEBDError
    wl = workloads.PARITY_L8
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt)
    g.set_option("randomized", 1)
    g.init_product(wl.occupation())
    with pytest.raises(TEBDError) as e:
        g.step(1)
    assert e.value.status == -4
    g.close()
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, u1=True)
    with pytest.raises(TEBDError):
        g.set_option("randomized", 1)
    g.close()
