"""The size-independent state checks, validated on oracle states and on planted defects."""
import numpy as np

import workloads
from oracle.tebd import TEBD
from state_checks import canonical_error, norm_error, particle_number


def _evolved(eps_rel=None):
    wl = workloads.TRUNC_L32
    o = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut,
             eps_rel=wl.eps_rel if eps_rel is None else eps_rel)
    o.init_product(wl.occupation())
    o.step(20)
    return o, int(wl.occupation().sum())


def test_checks_pass_on_an_untruncated_state():
    wl = workloads.PARITY_L8
    o = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=0.0, eps_rel=1e-24)
    o.init_product(wl.occupation())
    o.step(60)
    assert canonical_error(o.B) < 1e-13
    assert norm_error(o.lam) < 1e-14
    assert abs(particle_number(o.B, o.lam) - 4) < 1e-12


def test_truncated_state_keeps_norms_and_number():
    """With truncation (L = 32, w_cut = 1e-10) the bond vectors stay normalised and N moves at
    O(w_total); right-canonicality is only approximate there (see state_checks)."""
    o, N = _evolved()
    assert o.w_total > 0
    assert norm_error(o.lam) < 1e-14
    assert abs(particle_number(o.B, o.lam) - N) < max(1e-10, 10 * o.w_total)
    assert abs(particle_number(o.B, o.lam) - o.densities().sum()) < 1e-12


def test_checks_catch_planted_defects():
    o, N = _evolved(eps_rel=1e-24)
    B = [b.copy() for b in o.B]
    B[10] = 1.001 * B[10]
    assert canonical_error(B) > 1e-3
    lam = [x.copy() for x in o.lam]
    lam[16] = lam[16][::-1] * 1.0001
    assert norm_error(lam) > 1e-5
    B = [b.copy() for b in o.B]
    B[5] = np.roll(B[5], 1, axis=1)  # occupations shifted by one on site 5
    assert abs(particle_number(B, o.lam) - N) > 0.1


def test_checks_on_the_synthetic_saturated_state():
    B, lam, _ = workloads.synthetic_state(32, 4, 256)
    assert canonical_error(B) < 1e-12 and norm_error(lam) < 1e-14
