"""Parity at the headline size: L = 64, d = 5 (n_max = 4), chi_max = 1024, the
mixed-precision chain (U = 3, J_NNN = 0.1, K = 0.003 about j_c = 32.5, dt = 0.005).

The oracle cannot evolve this chain in seconds (one dense update of a saturated
triple takes minutes on the host), so:
  (a) one layer on the GPU from the charge-labelled saturated state; one interior
      triple of it through the U(1) oracle (the same update, one triple): the new
      spectra to 1e-10 and the densities of the three touched sites to 1e-9 on the
      FP64 and exact-digit paths, 1e-5 on the mixed path, max |delta| printed;
  (b) full steps on the GPU, then properties that hold at any size: every bond
      vector normalised, every bond sorted by charge with N on the last bond, each
      site tensor zero outside its charge blocks, the V2^+ tensors right-canonical;
  (c) the mixed and exact-digit paths against the FP64 path after the same full
      steps, max |dn_j| and |dcurrent| printed;
  (d) the dense path at the same local sizes (m = chi d = 5120 Gram matrices): the
      L = 16 chain with the same physics, whose middle bonds saturate at 1024, one
      layer, its middle triple against the dense oracle.
"""
import numpy as np
import pytest

import workloads
from oracle.tebd import TEBD as OracleTEBD
from oracle.u1 import U1TEBD
from state_checks import canonical_error, norm_error

pytestmark = pytest.mark.gpu

WL = workloads.MIXED_L64
N = 32  # half filling of the 64-site CDW
TRIPLE = 31  # 1-based first site of the interior triple checked (layer A: j = 1 mod 3)


def _args(wl, **kw):
    a = dict(L=wl.L, n_max=wl.n_max, chi_max=wl.chi_max, U=wl.U, J=wl.J, Jnnn=wl.Jnnn, K=wl.K, jc=wl.jc,
             dt=wl.dt, w_cut=wl.w_cut, eps_rel=wl.eps_rel)
    a.update(kw)
    return a


@pytest.fixture(scope="module")
def state_u1():
    return workloads.synthetic_state_u1(WL.L, WL.d, WL.chi_max, N)


@pytest.fixture(scope="module")
def oracle_triple(state_u1):
    B, lam, q = state_u1
    o = U1TEBD(**_args(WL))
    o.set_state(B, lam, q)
    i = TRIPLE - 1
    o.apply_gate(i, o.gate(TRIPLE, WL.dt / 2))
    n_o = o.densities()
    return {"n": n_o[i:i + 3].copy(), "lam1": np.sort(o.lam[i + 1])[::-1], "lam2": np.sort(o.lam[i + 2])[::-1],
            "q1": np.sort(o.q[i + 1]), "q2": np.sort(o.q[i + 2])}


def _gpu_u1(precision, state):
    from paper_2401_05301_gb300 import TEBD
    B, lam, q = state
    g = TEBD(**_args(WL), precision=precision, u1=True)
    g.set_state(B, lam)
    g.set_charges(q)
    return g


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (2, 1e-9), (1, 1e-5)])
def test_layer_interior_triple_matches_u1_oracle(lib, state_u1, oracle_triple, precision, tol):
    g = _gpu_u1(precision, state_u1)
    g.layer(0, False)
    n_g, _ = g.measure()
    i = TRIPLE - 1
    dn = float(np.max(np.abs(n_g[i:i + 3] - oracle_triple["n"])))
    l1 = np.sort(g.get_lambda(i + 1))[::-1]
    l2 = np.sort(g.get_lambda(i + 2))[::-1]
    assert len(l1) == len(oracle_triple["lam1"]) and len(l2) == len(oracle_triple["lam2"])
    dl = max(float(np.max(np.abs(l1 - oracle_triple["lam1"]))), float(np.max(np.abs(l2 - oracle_triple["lam2"]))))
    assert np.array_equal(np.sort(g.get_charges(i + 1)), oracle_triple["q1"])
    assert np.array_equal(np.sort(g.get_charges(i + 2)), oracle_triple["q2"])
    g.close()
    print(f"L64 d5 chi1024 triple {TRIPLE}, precision {precision}: max |dn| = {dn:.2e}, max |dlambda| = {dl:.2e}")
    assert dn < tol
    assert dl < (1e-10 if precision != 1 else 1e-5)


def _site_blocks_ok(B, ql, qr, d):
    allowed = qr[None, None, :] == ql[:, None, None] + np.arange(d)[None, :, None]
    return float(np.max(np.where(allowed, 0.0, np.abs(B)))) == 0.0


@pytest.fixture(scope="module")
def evolved(state_u1):
    """Two full steps (208 gate updates) on each path from the saturated state."""
    out = {}
    for precision in (0, 1, 2):
        g = _gpu_u1(precision, state_u1)
        g.step(2)
        n, cur = g.measure()
        out[precision] = (n, cur)
        if precision == 0:
            chi = g.bond_dims()
            Bs, lams, qs = [], [], []
            for k in range(WL.L + 1):
                qs.append(g.get_charges(k))
                if k < WL.L:
                    b, lm = g.get_site(k)
                    Bs.append(b)
                    lams.append(lm)
                else:
                    lams.append(g.get_lambda(k))
            out["state"] = (Bs, lams, qs, chi, g.stats())
        g.close()
    return out


def test_full_steps_keep_the_invariants(lib, evolved):
    """After full steps: every bond vector normalised; every bond sorted by charge with the
    chain's N on the last bond; each site tensor zero outside its blocks; and the tensors the
    last layer wrote as V2^+ (site i+2 of every triple i = 0 mod 3) right-canonical.  (The
    synthetic state's lambdas are not the Schmidt values of its tensors, so canonical-form
    densities of it need not sum to N.)"""
    Bs, lams, qs, chi, (t, w_total, max_chi) = evolved["state"]
    assert abs(t - 2 * WL.dt) < 1e-15 and max_chi == WL.chi_max
    assert norm_error(lams) < 1e-12
    for k in range(WL.L + 1):
        assert len(qs[k]) == chi[k] and np.all(np.diff(qs[k]) >= 0)
    assert list(qs[0]) == [0] and set(qs[WL.L]) == {N}
    for k in (0, 5, 30, 31, 32, 58, 63):
        assert _site_blocks_ok(Bs[k], qs[k], qs[k + 1], WL.d), f"site {k} has weight outside its blocks"
    ce = canonical_error([Bs[i + 2] for i in range(0, WL.L - 2, 3)])
    print(f"L64 after 2 steps: w_total = {w_total:.3e}, right-canonical error of the V2^+ sites = {ce:.2e}")
    # one Newton-Schulz step leaves rounding of order K eps (K <= 1024 kept rows)
    assert ce < 1e-11


def test_mixed_and_exact_paths_against_fp64(lib, evolved):
    n0, c0 = evolved[0]
    for precision, tol in ((1, 1e-5), (2, 1e-9)):
        n, c = evolved[precision]
        dn, dc = float(np.max(np.abs(n - n0))), float(np.max(np.abs(c - c0)))
        print(f"L64 d5 chi1024, 2 steps, precision {precision} vs FP64: max |dn| = {dn:.2e}, max |dcur| = {dc:.2e}")
        assert dn < tol and dc < tol


@pytest.mark.parametrize("precision,tol", [(0, 1e-9)])
def test_dense_path_saturated_triple(lib, precision, tol):
    """Dense path, m = chi d = 5120: the L = 16 chain of the same physics, whose bonds 5..11
    are saturated at 1024; one layer, its triple on sites 7..9 against the dense oracle."""
    from paper_2401_05301_gb300 import TEBD
    wl = workloads.SAMPLE_L16_D5
    B, lam, _ = workloads.synthetic_state(wl.L, wl.d, wl.chi_max)
    g = TEBD(**_args(wl), precision=precision)
    g.set_state(B, lam)
    g.layer(0, False)
    n_g, _ = g.measure()
    o = OracleTEBD(**_args(wl))
    o.set_state(B, lam)
    j = 7
    o.apply_gate(j - 1, o.gate(j, wl.dt / 2))
    n_o = o.densities()
    for b in (j, j + 1):
        lg, lo = g.get_lambda(b), o.lam[b]
        assert len(lg) == len(lo) == wl.chi_max
        assert np.max(np.abs(lg - lo)) < 1e-10
    dn = float(np.max(np.abs(n_g[j - 1:j + 2] - n_o[j - 1:j + 2])))
    g.close()
    print(f"dense L16 d5 chi1024 triple {j}: max |dn| = {dn:.2e}")
    assert dn < tol
