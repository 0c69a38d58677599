"""GPU super-site scheme (tebd_create_supersite: the paper's grouping of site pairs,
Sec. II B) against the super-site oracle, on the same seeded inputs.

The two sides take the same decomposition route (one SVD per two-site gate, the
B-form update), so densities, currents, chi' on every bond, sorted spectra and the
discarded weight are compared.  Bounds: 1e-9 on densities and currents for the FP64
(precision 0) and exact-digit (precision 2) paths, 1e-5 for the mixed path
(precision 1), 1e-10 on the spectra of every bond where chi' agrees (a bond
where it differs sits at a truncation tie and is reported).
"""
import numpy as np
import pytest

import workloads
from oracle.supersite import SuperSiteTEBD
from state_checks import canonical_error, norm_error

pytestmark = pytest.mark.gpu

TOL = 1e-9
TOL_MIXED = 1e-5


def _args(wl, **kw):
    a = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
             dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    a.update(kw)
    return a


def _gpu(wl, precision=0, **kw):
    from paper_2401_05301_gb300 import SuperSiteTEBD as GpuSS
    return GpuSS(**_args(wl, **kw), precision=precision)


def _check_bonds(g, o, spectra_tol=1e-10):
    chi_g, chi_o = list(g.bond_dims()), o.chi()
    differ = [k for k, (a, b) in enumerate(zip(chi_g, chi_o)) if a != b]
    for k in range(g.L + 1):
        if k in differ:
            continue
        lg, lo = np.sort(g.get_lambda(k))[::-1], np.sort(o.lam[k])[::-1]
        assert np.max(np.abs(lg - lo)) < spectra_tol, (k, np.max(np.abs(lg - lo)))
    return differ


def _compare_run(wl, n_steps, every, precision=0, tol=TOL, spectra=True):
    g = _gpu(wl, precision)
    o = SuperSiteTEBD(**_args(wl))
    occ = wl.occupation()
    g.init_product(occ)
    o.init_product(occ)
    worst = 0.0
    for k in range(every, n_steps + 1, every):
        g.step(every)
        o.step(every)
        n_g, cur_g = g.measure()
        assert n_g.shape == (o.Lp,) and cur_g.shape == (o.Lp - 1,)
        err = max(np.max(np.abs(n_g - o.densities())), np.max(np.abs(cur_g - o.currents())))
        differ = _check_bonds(g, o) if spectra else []
        assert err < tol, f"step {k}: max |dn|,|dcur| = {err:.3e}; chi' differs on bonds {differ}"
        if differ:
            print(f"step {k}: chi' differs on bonds {differ} (a truncation tie); observables still within bound")
        worst = max(worst, err)
    t, w, _ = g.stats()
    assert abs(t - n_steps * wl.dt) < 1e-12
    assert abs(w - o.w_total) <= 1e-9 * max(1.0, o.w_total) + 1e-14
    g.close()
    return worst


def test_supersite_product_state(lib):
    """The product state maps physical pairs to sigma = s_a d + s_b; an odd chain's padded
    site is empty."""
    wl = workloads.Workload("ss7", L=7, n_max=2, chi_max=16, U=2.0, J=1.0, Jnnn=0.2, K=0.0, jc=4.0, dt=0.05,
                            t_end=0.5)
    g = _gpu(wl)
    occ = np.array([2, 0, 1, 1, 0, 2, 1])
    g.init_product(occ)
    n, cur = g.measure()
    assert np.array_equal(n, np.append(occ, 0).astype(float))
    assert np.all(cur == 0.0)
    assert g.L == 4 and list(g.bond_dims()) == [1] * 5
    B, _ = g.get_site(1)
    assert B.shape == (1, 9, 1) and B[0, 1 * 3 + 1, 0] == 1.0
    g.close()


@pytest.mark.parametrize("L,n_max,chi", [(7, 2, 81), (8, 1, 16), (3, 3, 16), (4, 1, 1), (9, 2, 5)])
def test_supersite_small_chains(lib, L, n_max, chi):
    """Odd and even chains, the smallest (one super bond), chi = 1 and a tight cap."""
    wl = workloads.Workload("ss", L=L, n_max=n_max, chi_max=chi, U=2.0, J=1.0, Jnnn=0.25, K=0.03,
                            jc=(L + 1) / 2, dt=0.05, t_end=1.0, w_cut=1e-10)
    worst = _compare_run(wl, 20, 5)
    print(f"supersite L{L} n_max{n_max} chi{chi}: max |delta| = {worst:.3e}")


def test_supersite_truncating_chain(lib):
    """L = 20, d_e = 16, chi_max = 32, w_cut = 1e-10: the cap binds in the middle."""
    wl = workloads.Workload("ss20", L=20, n_max=3, chi_max=32, U=4.0, J=1.0, Jnnn=0.12, K=0.005, jc=10.5,
                            dt=0.02, t_end=1.0, w_cut=1e-10)
    worst = _compare_run(wl, 30, 10)
    print(f"supersite L20 truncating: max |delta| = {worst:.3e}")


@pytest.mark.parametrize("precision,tol", [(2, TOL), (1, TOL_MIXED)])
def test_supersite_precisions(lib, precision, tol):
    wl = workloads.Workload("ss12", L=12, n_max=2, chi_max=64, U=3.0, J=1.0, Jnnn=0.1, K=0.01, jc=6.5,
                            dt=0.02, t_end=1.0, w_cut=1e-12)
    worst = _compare_run(wl, 20, 10, precision=precision, tol=tol, spectra=(precision != 1))
    print(f"supersite precision {precision}: max |delta| = {worst:.3e} (bound {tol:g})")


def test_supersite_paper_setup_flanked_cdw(lib):
    """The paper's run: L = 121 padded to 122 (61 super sites, d_e = 25), flanked CDW of
    27 bosons, Table Ib set a, dt = 0.05 pi/2, chi_max = 40; five steps, every step."""
    worst = _compare_run(workloads.paper_run("a", 27, 40), 5, 1)
    print(f"supersite paper setup chi40: max |delta| = {worst:.3e}")


def _synthetic_layer(wl, L_e, bonds_checked):
    """A saturated synthetic super-site state; one odd layer (dt/2) on the GPU; the same
    gates on the checked bonds (0-based i, even) through the oracle."""
    from paper_2401_05301_gb300 import SuperSiteTEBD as GpuSS
    de = (wl.n_max + 1) ** 2
    B, lam, chi = workloads.synthetic_state(L_e, de, wl.chi_max)
    g = GpuSS(**_args(wl))
    g.set_state(B, lam)
    g.layer(0, False)
    n_g, cur_g = g.measure()
    o = SuperSiteTEBD(**_args(wl))
    o.B = [b.copy() for b in B]
    o.lam = [x.copy() for x in lam]
    worst = 0.0
    for i in bonds_checked:
        o.apply_gate(i, o.gate(i + 1, wl.dt / 2))
    n_o, cur_o = o.densities(), o.currents()
    for i in bonds_checked:
        lg, lo = g.get_lambda(i + 1), o.lam[i + 1]
        assert len(lg) == len(lo)
        assert np.max(np.abs(np.sort(lg)[::-1] - np.sort(lo)[::-1])) < 1e-10
        sites = slice(2 * i, 2 * i + 4)
        worst = max(worst, float(np.max(np.abs(n_g[sites] - n_o[sites]))),
                    float(np.max(np.abs(cur_g[2 * i:2 * i + 3] - cur_o[2 * i:2 * i + 3]))))
    # the layer wrote B_{i+1} = V^+ of every odd bond: right-canonical
    ce = canonical_error([g.get_site(i + 1)[0] for i in range(0, L_e - 1, 2)])
    lams = [g.get_lambda(k) for k in range(L_e + 1)]
    g.close()
    return worst, ce, norm_error(lams)


def test_supersite_synthetic_layer_chi40(lib):
    """61 super sites of d_e = 25 saturated at chi = 40 (theta' of 1000 x 1000), every odd
    bond through the oracle."""
    wl = workloads.paper_run("a", 27, 40)
    worst, ce, ne = _synthetic_layer(wl, 61, list(range(0, 60, 2)))
    print(f"supersite synthetic chi40 layer: max |delta| = {worst:.3e}, canonical {ce:.2e}")
    assert worst < TOL and ce < 1e-12 and ne < 1e-12


def test_supersite_synthetic_layer_chi200(lib):
    """8 super sites of d_e = 25 saturated at chi = 200 (theta' of 5000 x 5000), the
    middle odd bond through the oracle."""
    wl = workloads.Workload("ss16_chi200", L=16, n_max=4, chi_max=200, U=2.442, J=1.0, Jnnn=-0.12, K=0.01,
                            jc=8.5, dt=0.05 * np.pi / 2, t_end=1.0, w_cut=1e-12)
    worst, ce, ne = _synthetic_layer(wl, 8, [2])
    print(f"supersite synthetic chi200 layer: max |delta| = {worst:.3e}, canonical {ce:.2e}")
    assert worst < TOL and ce < 1e-11 and ne < 1e-12


def test_supersite_refusals(lib):
    from paper_2401_05301_gb300 import SuperSiteTEBD as GpuSS, TEBD, TEBDError, batch_step
    import ctypes
    from paper_2401_05301_gb300 import binding
    g = GpuSS(8, 2, 16, 2.0, 1.0, 0.1, 0.0, 4.5, 0.01)
    for key, val in (("u1", 1), ("randomized", 1), ("trotter_order", 4)):
        with pytest.raises(TEBDError) as e:
            g.set_option(key, val)
        assert e.value.status == -1
    g.init_product(workloads.cdw(8))
    with pytest.raises(TEBDError):
        g.layer(2, False)
    with pytest.raises(TEBDError):
        g.init_product(np.array([3, 0, 0, 0, 0, 0, 0, 0]))  # above n_max
    t = TEBD(8, 2, 16, 2.0, 1.0, 0.1, 0.0, 4.5, 0.01)
    t.init_product(workloads.cdw(8))
    with pytest.raises(TEBDError):
        batch_step([g, t], 1)
    h = ctypes.c_void_p()
    assert binding.load().tebd_create_supersite(8, 5, 16, 2.0, 1.0, 0.1, 0.0, 4.5, 0.01, ctypes.byref(h)) == -1
    assert not h.value
    g.close()
    t.close()


def test_supersite_batch_is_bitwise_the_same_as_alone(lib):
    from paper_2401_05301_gb300 import SuperSiteTEBD as GpuSS, batch_step
    sims = [(9, 2, 32, 2.0, 1.0, 0.1, 0.01, 5.0, 0.02, 1e-10), (12, 1, 16, 5.0, 1.0, 0.12, 0.005, 6.5, 0.01, 0.0),
            (6, 3, 64, 3.0, 1.0, 0.05, 0.0, 3.5, 0.01, 0.0)]

    def make(p):
        L, n_max, chi, U, J, Jnnn, K, jc, dt, wc = p
        g = GpuSS(L, n_max, chi, U, J, Jnnn, K, jc, dt, w_cut=wc)
        g.init_product(workloads.cdw(L))
        return g

    alone = []
    for p in sims:
        g = make(p)
        g.step(12)
        alone.append(np.concatenate(g.measure()))
        g.close()
    hs = [make(p) for p in sims]
    for _ in range(3):
        batch_step(hs, 4)
    for g, ref in zip(hs, alone):
        assert np.array_equal(np.concatenate(g.measure()), ref)
        g.close()
