"""CUDA-graph replay of whole steps (option "graph", dense three-site form).

A replay is accepted only when every host decision it fixed in advance (all kmax
eigenvectors, chi' equal to each bond's capacity) is confirmed on the device, so
an accepted step performs exactly the kernels of the ordinary step with the same
arguments: the results must be bitwise those of the ordinary path.  A replay
that is undone (here forced by the "graph_test_fallback" diagnostic) restores
the state from the graph's own backup and runs the step the ordinary way, so it
too ends bitwise equal.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

L, N_MAX, CHI = 16, 3, 64  # d = 4: bonds 3..13 saturated at chi = 64 in the synthetic state
PHYS = dict(U=5.0, J=1.0, Jnnn=0.12, K=0.005, jc=8.5, dt=0.01)


def _make(precision=0, graph=False, **kw):
    from paper_2401_05301_gb300 import TEBD
    g = TEBD(L, N_MAX, CHI, PHYS["U"], PHYS["J"], PHYS["Jnnn"], PHYS["K"], PHYS["jc"], PHYS["dt"],
             precision=precision, **kw)
    B, lam, _ = workloads.synthetic_state(L, N_MAX + 1, CHI)
    g.set_state(B, lam)
    if graph:
        g.set_option("graph", 1)
    return g


def _snapshot(g):
    chi = g.bond_dims()
    sites = [g.get_site(k) for k in range(L)]
    n, cur = g.measure()
    return chi, sites, g.get_lambda(L), n, cur, g.stats()


def _assert_bitwise(a, b):
    chi_a, sites_a, lamL_a, n_a, c_a, st_a = a
    chi_b, sites_b, lamL_b, n_b, c_b, st_b = b
    assert np.array_equal(chi_a, chi_b)
    for (Ba, la), (Bb, lb) in zip(sites_a, sites_b):
        assert np.array_equal(Ba, Bb) and np.array_equal(la, lb)
    assert np.array_equal(lamL_a, lamL_b)
    assert np.array_equal(n_a, n_b) and np.array_equal(c_a, c_b)
    assert st_a == st_b


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_graph_steps_are_bitwise_the_ordinary_steps(lib, precision):
    ref = _make(precision)
    ref.step(5)
    g = _make(precision, graph=True)
    g.step(5)  # step 1 ordinary, step 2 captured and replayed, steps 3-5 replayed
    replays, fallbacks, per = g.graph_stats()
    print(f"precision {precision}: {replays} replays, {fallbacks} undone, {per} launches per replay")
    assert replays == 4 and fallbacks == 0 and per > 0
    _assert_bitwise(_snapshot(g), _snapshot(ref))
    g.close()
    ref.close()


def test_undone_replay_restores_and_reruns(lib):
    ref = _make(0)
    ref.step(4)
    g = _make(0, graph=True)
    g.step(2)
    g.set_option("graph_test_fallback", 1)
    g.step(2)  # the first of these replays is undone and rerun the ordinary way
    replays, fallbacks, _ = g.graph_stats()
    assert fallbacks == 1 and replays >= 1
    _assert_bitwise(_snapshot(g), _snapshot(ref))
    g.close()
    ref.close()


def test_batched_graph_steps(lib):
    from paper_2401_05301_gb300 import batch_step
    refs = [_make(1) for _ in range(3)]
    hs = [_make(1, graph=(i == 0)) for i in range(3)]  # the driving handle holds the option
    for g in hs[1:]:
        g.set_option("graph", 1)
    for _ in range(4):
        batch_step(refs, 1)
        batch_step(hs, 1)
    replays, fallbacks, per = hs[0].graph_stats()
    assert replays == 3 and fallbacks == 0 and per > 0
    for g, r in zip(hs, refs):
        _assert_bitwise(_snapshot(g), _snapshot(r))
        g.close()
        r.close()


def test_graph_not_used_below_capacity(lib):
    """A chain that is not saturated (a product state) runs the ordinary path; the
    option is refused where it cannot be exact."""
    from paper_2401_05301_gb300 import TEBD, TEBDError
    g = TEBD(L, N_MAX, CHI, PHYS["U"], PHYS["J"], PHYS["Jnnn"], PHYS["K"], PHYS["jc"], PHYS["dt"])
    g.set_option("graph", 1)
    g.init_product(workloads.cdw(L))
    g.step(3)
    assert g.graph_stats()[0] == 0
    g.close()
    u = TEBD(L, N_MAX, CHI, PHYS["U"], PHYS["J"], PHYS["Jnnn"], PHYS["K"], PHYS["jc"], PHYS["dt"], u1=True)
    with pytest.raises(TEBDError):
        u.set_option("graph", 1)
    u.close()
