"""Input builders: the flanked CDW of the paper's setup (Sec. II C) and its parameter sets."""
import numpy as np
import pytest

import workloads


def test_flanked_cdw_matches_sec_2c():
    """L = 121, N = 27: the middle site (the paper's j = 0) is occupied, sites at odd
    distance from it are empty, 27 bosons fill j = -26..26 and the flanks are empty."""
    occ = workloads.flanked_cdw(121, 27)
    j = np.arange(121) - 60  # the paper's index, j = 0 in the middle, |j| <= 60
    assert occ.sum() == 27
    assert np.array_equal(np.flatnonzero(occ), np.flatnonzero((np.abs(j) <= 26) & (j % 2 == 0)))
    assert np.array_equal(occ, occ[::-1])
    for N in (3, 43):  # the paper's range of odd N
        o = workloads.flanked_cdw(121, N)
        assert o.sum() == N and o[60] == 1 and o[59] == 0


@pytest.mark.parametrize("L,N", [(120, 27), (121, 26), (11, 7), (5, 0)])
def test_flanked_cdw_rejects_bad_shapes(L, N):
    with pytest.raises(ValueError):
        workloads.flanked_cdw(L, N)


def test_paper_run_setup():
    wl = workloads.paper_run("c", 27, 1000)
    assert (wl.L, wl.d, wl.chi_max, wl.n_steps, wl.measure_every) == (121, 5, 1000, 100, 1)
    assert wl.dt == pytest.approx(0.05 * np.pi / 2, rel=1e-15)
    assert (wl.U, wl.Jnnn, wl.K, wl.J, wl.jc) == (5.167, -0.05, 0.017, 1.0, 61.0)
    assert wl.w_cut == wl.eps_rel == 1e-12
    assert wl.occupation()[60] == 1 and wl.occupation().sum() == 27
    assert wl.n_steps * wl.dt == pytest.approx(2.5 * np.pi)  # t = 5 pi/2, the paper's last time


def test_paper_params_match_table_1b():
    """workloads.PAPER_PARAMS against the printed Table I(b) (tests/golden): a flipped J_NNN sign
    or swapped columns would fail here."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table_1b_parameters.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert [r[0] for r in rows] == ["a", "b", "c", "d"]
    for sim, U, Jnnn, K, J in rows:
        assert workloads.PAPER_PARAMS[sim] == (float(U), float(Jnnn), float(K))
        assert float(J) == 1.0 == workloads.paper_run(sim, 27, 40).J
