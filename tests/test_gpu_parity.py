"""GPU FP64 path vs the CPU oracle, element by element on the same seeded inputs.

Tolerance 1e-9 on densities and currents (the stated FP64 parity bound);
truncation decisions are compared too: a differing kept count chi' is
reported with the smallest gap at the cut rather than hidden.
"""
import numpy as np
import pytest

import workloads
from oracle.tebd import TEBD as OracleTEBD

pytestmark = pytest.mark.gpu

TOL = 1e-9


def _pair(lib, wl, precision=None, **kw):
    from paper_2401_05301_gb300 import TEBD
    args = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
                dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    args.update(kw)
    g = TEBD(**args, precision=precision)
    o = OracleTEBD(**args)
    return g, o


def _compare_run(lib, wl, n_steps, every, **kw):
    g, o = _pair(lib, wl, **kw)
    occ = wl.occupation()
    g.init_product(occ)
    o.init_product(occ)
    worst = 0.0
    for k in range(every, n_steps + 1, every):
        g.step(every)
        o.step(every)
        n_g, cur_g = g.measure()
        n_o, cur_o = o.densities(), o.currents()
        err = max(np.max(np.abs(n_g - n_o)), np.max(np.abs(cur_g - cur_o)))
        chi_g, chi_o = list(g.bond_dims()), o.chi()
        differ = sum(int(a != b) for a, b in zip(chi_g, chi_o))
        assert err < TOL, (f"step {k}: max |dn|,|dcur| = {err:.3e}; chi' differs on {differ} bonds "
                           f"(gpu {chi_g} oracle {chi_o}); smallest relative gap at a cut so far "
                           f"{o.min_cut_gap:.2e}" + ("  -> unpinned at a truncation tie" if differ else ""))
        worst = max(worst, err)
    print(f"{wl.name}: smallest relative gap at a truncation cut {o.min_cut_gap:.2e}")
    t, w, _ = g.stats()
    assert abs(t - n_steps * wl.dt) < 1e-12
    assert abs(w - o.w_total) <= 1e-9 * max(1.0, o.w_total) + 1e-14
    g.close()
    return worst


def test_small_chain_matches_oracle(lib):
    wl = workloads.Workload("small", L=6, n_max=2, chi_max=64, U=2.0, J=1.0, Jnnn=0.2, K=0.05, jc=3.5,
                            dt=0.05, t_end=1.0)
    _compare_run(lib, wl, 20, 5)


def test_parity_L8_full_trajectory(lib):
    """L=8, d=4, N=4, chi_max=256 (untruncated up to the paper's eps), t = 0..4 every 0.1."""
    wl = workloads.PARITY_L8
    worst = _compare_run(lib, wl, wl.n_steps, wl.measure_every)
    print(f"L8 parity: max |delta| = {worst:.3e}")


def test_parity_L32_truncating(lib):
    """L=32, d=4, w_cut = 1e-10, to t = 1 (the oracle's seconds-scale prefix)."""
    wl = workloads.TRUNC_L32
    worst = _compare_run(lib, wl, 100, 10)
    print(f"L32 parity: max |delta| = {worst:.3e}")


def test_paper_setup_flanked_cdw(lib):
    """The paper's own setup (Sec. II C): L = 121, d = 5, flanked CDW of 27 bosons,
    Table Ib set a (J_NNN < 0), dt = 0.05 pi/2, cuts w = eps = 1e-12, chi_max = 40
    (the paper's smallest); eight steps, measured every second step."""
    worst = _compare_run(lib, workloads.paper_run("a", 27, 40), 8, 2)
    print(f"paper setup parity: max |delta| = {worst:.3e}")


@pytest.mark.parametrize("name,steps,every", [("PARITY_L8", 400, 10), ("TRUNC_L32", 100, 10)])
def test_exact_digit_precision_holds_fp64_bound(lib, name, steps, every):
    """precision 2: every large product (contractions, Gram, projection, reduction
    updates, back-transformation) on the exact-digit tensor-core engine; the FP64
    parity bound must still hold."""
    worst = _compare_run(lib, getattr(workloads, name), steps, every, precision=2)
    print(f"{name} exact-digit parity: max |delta| = {worst:.3e}")


def test_fourth_order_split_matches_oracle(lib):
    """trotter_order 4 (Suzuki's composition of the second-order step, 25 layers):
    the GPU FP64 path against the oracle's fourth-order split, L=8, to t = 0.6."""
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.PARITY_L8
    args = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
                dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    g = TEBD(**args)
    g.set_option("trotter_order", 4)
    o = OracleTEBD(**args, order=4)
    occ = wl.occupation()
    g.init_product(occ)
    o.init_product(occ)
    worst = 0.0
    for _ in range(6):
        g.step(10)
        o.step(10)
        n_g, cur_g = g.measure()
        worst = max(worst, np.max(np.abs(n_g - o.densities())), np.max(np.abs(cur_g - o.currents())))
    t, _, _ = g.stats()
    g.close()
    print(f"fourth-order parity: max |delta| = {worst:.3e}")
    assert abs(t - 60 * wl.dt) < 1e-12
    assert worst < TOL


def test_hard_core_free_fermions_on_gpu(lib):
    """n_max = 1, J_NNN = 0: the GPU run follows the Trotterised free-fermion propagator.

    The Gram route resolves singular values down to p ~ 1e-15; the oracle run
    with the same floor deviates from the free propagator by ~1e-8..1e-7 here
    (discarded components grow like sqrt(p)), so the bound is 5e-7."""
    from oracle import free
    from paper_2401_05301_gb300 import TEBD
    L, dt, steps = 16, 0.02, 50
    g = TEBD(L, 1, 256, 7.0, 1.0, 0.0, 0.01, 8.5, dt, eps_rel=1e-15)
    occ = workloads.cdw(L)
    g.init_product(occ)
    g.step(steps)
    n_g, cur_g = g.measure()
    n, C = free.observables(free.trotter_propagator(L, 1.0, 0.0, 0.01, 8.5, dt, steps), occ)
    err = max(np.max(np.abs(n_g - n)), np.max(np.abs(cur_g - 2 * C.imag)))
    print(f"hard-core vs free fermions: {err:.2e}")
    assert err < 5e-7


@pytest.mark.parametrize("L,n_max,chi", [(3, 3, 64), (4, 1, 4), (5, 2, 1), (7, 2, 3), (9, 3, 5)])
def test_edge_shapes(lib, L, n_max, chi):
    """Single triple (L=3), d=2, chi_max=1 (stays a product state), heavy truncation."""
    wl = workloads.Workload("edge", L=L, n_max=n_max, chi_max=chi, U=1.5, J=1.0, Jnnn=0.3, K=0.02,
                            jc=(L + 1) / 2, dt=0.05, t_end=0.5, w_cut=1e-8)
    _compare_run(lib, wl, 10, 5)


def test_zero_steps_and_argument_errors(lib):
    from paper_2401_05301_gb300 import TEBD, TEBDError
    g = TEBD(6, 2, 16, 1.0, 1.0, 0.1, 0.0, 3.5, 0.01)
    with pytest.raises(TEBDError):
        g.step(1)  # before init
    g.init_product([1, 0, 1, 0, 1, 0])
    g.step(0)
    n, cur = g.measure()
    assert np.allclose(n, [1, 0, 1, 0, 1, 0]) and np.allclose(cur, 0)
    with pytest.raises(TEBDError):
        g.init_product([3, 0, 0, 0, 0, 0])  # occupation > n_max
    with pytest.raises(TEBDError):
        g.set_option("nope", 1.0)
    with pytest.raises(TEBDError):
        g.layer(3, True)
    with pytest.raises(TEBDError):
        TEBD(2, 2, 16, 1.0, 1.0, 0.1, 0.0, 3.5, 0.01)
    with pytest.raises(TEBDError):
        TEBD(6, 2, 16, 1.0, 1.0, 0.1, 0.0, 3.5, -0.01)


def test_bitwise_reproducible(lib):
    wl = workloads.TRUNC_L32
    outs = []
    for _ in range(2):
        from paper_2401_05301_gb300 import TEBD
        g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut)
        g.init_product(wl.occupation())
        g.step(30)
        outs.append(np.concatenate(g.measure()))
        g.close()
    assert np.array_equal(outs[0], outs[1])


def test_full_size_layer_sampled(lib):
    """Bench-size synthetic saturated state (L=32, d=4, chi=256): one A layer on the GPU
    vs the oracle on three sampled triples; compare the new bond spectra and the
    densities of the touched sites."""
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.TRUNC_L32
    B, lam, chi = workloads.synthetic_state(wl.L, wl.d, wl.chi_max)
    g = TEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut)
    g.set_state(B, lam)
    g.layer(0, False)
    n_g, _ = g.measure()
    o = OracleTEBD(wl.L, wl.n_max, wl.chi_max, wl.U, wl.J, wl.Jnnn, wl.K, wl.jc, wl.dt, w_cut=wl.w_cut)
    o.set_state(B, lam)
    for j in (1, 13, 25):  # triples in layer A (j = 1 mod 3), left edge and interior
        o.apply_gate(j - 1, o.gate(j, wl.dt / 2))
        for b in (j, j + 1):
            lg = g.get_lambda(b)
            lo = o.lam[b]
            assert len(lg) == len(lo), (j, b, len(lg), len(lo))
            assert np.max(np.abs(lg - lo)) < 1e-10
        # densities of the triple's sites depend only on this triple's update
        n_o = o.densities()
        for site in (j - 1, j, j + 1):
            assert abs(n_g[site] - n_o[site]) < TOL
