"""Failure statuses on the GPU, each produced without a GPU fault.

* TEBD_ERR_TIMEOUT: the handle's "wait_limit_clocks" option shortens every
  grid-barrier wait of the cooperative tridiagonal reduction to zero ticks, so
  the first barrier of the first panel runs out; the blocks record the failure
  and leave, the step returns the status, the handle stays in it (sticky), and
  a fresh handle on the same context still matches the oracle.
* TEBD_ERR_NONFINITE: a NaN installed in one lambda through tebd_set_state
  reaches the Gram trace of the triple that reads it; the step refuses it.
* TEBD_ERR_NOT_CONVERGED: a host Jacobi sweep limit of 1 for the gate table.
"""
import numpy as np
import pytest

import workloads
from oracle.tebd import TEBD as OracleTEBD

pytestmark = pytest.mark.gpu


def _handle(wl, **kw):
    from paper_2401_05301_gb300 import TEBD
    return TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut,
                eps_rel=wl.eps_rel, **kw)


def _still_works(lib):
    wl = workloads.Workload("after", L=6, n_max=2, chi_max=32, U=2.0, J=1.0, Jnnn=0.2, K=0.05, jc=3.5,
                            dt=0.05, t_end=0.5)
    g = _handle(wl)
    g.init_product(wl.occupation())
    g.step(5)
    n, cur = g.measure()
    g.close()
    o = OracleTEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut,
                   eps_rel=wl.eps_rel)
    o.init_product(wl.occupation())
    o.step(5)
    assert max(np.max(np.abs(n - o.densities())), np.max(np.abs(cur - o.currents()))) < 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_barrier_wait_that_runs_out_reports_timeout(lib, precision):
    from paper_2401_05301_gb300 import TEBDError
    wl = workloads.TRUNC_L32
    B, lam, _ = workloads.synthetic_state(wl.L, wl.d, wl.chi_max)
    g = _handle(wl, precision=precision)
    g.set_state(B, lam)
    g.set_option("wait_limit_clocks", 0)
    with pytest.raises(TEBDError) as e:
        g.step(1)
    assert e.value.status == -6
    with pytest.raises(TEBDError) as e2:  # sticky
        g.measure()
    assert e2.value.status == -6
    g.close()
    _still_works(lib)


def test_nan_lambda_reports_nonfinite(lib):
    from paper_2401_05301_gb300 import TEBDError
    wl = workloads.TRUNC_L32
    B, lam, _ = workloads.synthetic_state(wl.L, wl.d, wl.chi_max)
    lam = [x.copy() for x in lam]
    lam[3][0] = float("nan")  # left bond of the triple on sites 4..6 (1-based), in the first layer
    g = _handle(wl)
    g.set_state(B, lam)
    with pytest.raises(TEBDError) as e:
        g.step(1)
    assert e.value.status == -7
    with pytest.raises(TEBDError) as e2:
        g.step(1)
    assert e2.value.status == -7
    g.close()
    _still_works(lib)


def test_jacobi_sweep_limit_reports_not_converged(lib):
    from paper_2401_05301_gb300 import TEBDError
    wl = workloads.PARITY_L8
    g = _handle(wl)
    with pytest.raises(TEBDError) as e:
        g.set_option("jacobi_max_sweeps", 1)
    assert e.value.status == -5
    with pytest.raises(TEBDError) as e2:  # sticky
        g.init_product(wl.occupation())
    assert e2.value.status == -5
    g.close()
