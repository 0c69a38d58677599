"""Thin ctypes binding of libptebd.so (argument marshalling only).

Every step of the TEBD path runs inside the library's CUDA kernels; this
module converts Python/numpy arguments to the C ABI declared in
``include/ptebd.h`` and raises on non-zero status.  There is no fallback: if
the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptebd.so")

_c_int, _c_double, _c_void_p = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_P_int = ctypes.POINTER(ctypes.c_int)
_P_double = ctypes.POINTER(ctypes.c_double)
_P_ll = ctypes.POINTER(ctypes.c_longlong)

# void (*)(long long call, int n, int l, double* out, void* ctx): the randomized truncation's test matrices
TEST_MATRIX_FN = ctypes.CFUNCTYPE(None, ctypes.c_longlong, _c_int, _c_int, _P_double, _c_void_p)

# name -> (restype, argtypes); mirrors include/ptebd.h
SIGNATURES = {
    "tebd_create": (_c_int, [_c_int, _c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double,
                             _c_double, ctypes.POINTER(_c_void_p)]),
    "tebd_create_supersite": (_c_int, [_c_int, _c_int, _c_int, _c_double, _c_double, _c_double, _c_double,
                                       _c_double, _c_double, ctypes.POINTER(_c_void_p)]),
    "tebd_set_option": (_c_int, [_c_void_p, ctypes.c_char_p, _c_double]),
    "tebd_set_stream": (_c_int, [_c_void_p, _c_void_p]),
    "tebd_init_product": (_c_int, [_c_void_p, _P_int]),
    "tebd_step": (_c_int, [_c_void_p, _c_int]),
    "tebd_layer": (_c_int, [_c_void_p, _c_int, _c_int]),
    "tebd_batch_step": (_c_int, [ctypes.POINTER(_c_void_p), _c_int, _c_int]),
    "tebd_estimate_bytes": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _P_double]),
    "tebd_estimate_bytes_u1": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _P_double]),
    "tebd_measure": (_c_int, [_c_void_p, _P_double, _P_double]),
    "tebd_stats": (_c_int, [_c_void_p, _P_double, _P_double, _P_int]),
    "tebd_device_bytes": (_c_int, [_c_void_p, _P_double]),
    "tebd_bond_dims": (_c_int, [_c_void_p, _P_int]),
    "tebd_get_site": (_c_int, [_c_void_p, _c_int, _P_double, _P_double]),
    "tebd_set_state": (_c_int, [_c_void_p, _P_int, ctypes.POINTER(_P_double), ctypes.POINTER(_P_double)]),
    "tebd_set_charges": (_c_int, [_c_void_p, ctypes.POINTER(_P_int)]),
    "tebd_set_test_matrices": (_c_int, [_c_void_p, TEST_MATRIX_FN, _c_void_p]),
    "tebd_get_charges": (_c_int, [_c_void_p, _c_int, _P_int]),
    "tebd_counters": (_c_int, [_c_void_p, _P_ll, _P_ll]),
    "tebd_graph_stats": (_c_int, [_c_void_p, _P_ll, _P_ll, _P_ll]),
    "tebd_profile": (_c_int, [_c_void_p, _c_int, _P_double, _P_ll, _P_double]),
    "tebd_destroy": (None, [_c_void_p]),
    "tebd_strerror": (ctypes.c_char_p, [_c_int]),
    "tebd_zgemm": (_c_int, [_c_int, _c_int, _c_int, _c_int, _c_int, _c_double, _c_void_p, ctypes.c_longlong,
                            _c_void_p, ctypes.c_longlong, _c_void_p, ctypes.c_longlong, _c_void_p]),
    "tebd_bond_correlator_noalloc": (_c_int, [_c_void_p, _c_void_p, _c_void_p, _c_int, _c_int, _c_int, _c_int,
                                             _c_void_p, _c_void_p]),
    "tebd_gate_host": (_c_int, [_c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double, _c_int,
                                _c_double, _P_double]),
    "tebd_gate_host_sweeps": (_c_int, [_c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double,
                                       _c_int, _c_double, _c_int, _P_double]),
    "tebd_gate_host_supersite": (_c_int, [_c_int, _c_int, _c_double, _c_double, _c_double, _c_double, _c_double,
                                          _c_int, _c_double, _P_double]),
}

_LIB = None


class TEBDError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = load().tebd_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def load():
    """Load libptebd.so (built in-tree) and declare its signatures."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libptebd.so is not built: run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int, where: str):
    if status != 0:
        raise TEBDError(status, where)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_P_double)


def estimate_bytes(L, n_max, chi_max, max_slots=0, precision=0, u1=False) -> float:
    """Device bytes a simulation of these sizes will hold (tebd_estimate_bytes, or
    tebd_estimate_bytes_u1 for the particle-number-blocked form)."""
    out = _c_double()
    if u1:
        _check(load().tebd_estimate_bytes_u1(L, n_max, chi_max, max_slots, precision, ctypes.byref(out)),
               "tebd_estimate_bytes_u1")
    else:
        _check(load().tebd_estimate_bytes(L, n_max, chi_max, max_slots, precision, ctypes.byref(out)),
               "tebd_estimate_bytes")
    return out.value


def batch_step(sims, n_steps: int = 1):
    """Advance several TEBD handles together (tebd_batch_step)."""
    arr = (_c_void_p * len(sims))(*[s._h for s in sims])
    _check(load().tebd_batch_step(arr, len(sims), int(n_steps)), "tebd_batch_step")


def gate_host(L, n_max, U, J, Jnnn, K, jc, j, tau) -> np.ndarray:
    """The library's host-built gate exp(-i h_j tau), d^3 x d^3 complex."""
    d = n_max + 1
    out = np.empty(2 * d ** 6, dtype=np.float64)
    _check(load().tebd_gate_host(L, n_max, U, J, Jnnn, K, jc, j, tau, _dptr(out)), "tebd_gate_host")
    return out.view(np.complex128).reshape(d ** 3, d ** 3)


def gate_host_sweeps(L, n_max, U, J, Jnnn, K, jc, j, tau, max_sweeps) -> np.ndarray:
    """tebd_gate_host with a sweep limit for the host Jacobi solver; raises TEBDError
    (status TEBD_ERR_NOT_CONVERGED) when the solver did not converge in time."""
    d = n_max + 1
    out = np.empty(2 * d ** 6, dtype=np.float64)
    _check(load().tebd_gate_host_sweeps(L, n_max, U, J, Jnnn, K, jc, j, tau, int(max_sweeps), _dptr(out)),
           "tebd_gate_host_sweeps")
    return out.view(np.complex128).reshape(d ** 3, d ** 3)


def gate_host_supersite(L, n_max, U, J, Jnnn, K, jc, k, tau) -> np.ndarray:
    """The library's host-built gate exp(-i h_k tau) of super bond k, d^4 x d^4 complex."""
    d = n_max + 1
    out = np.empty(2 * d ** 8, dtype=np.float64)
    _check(load().tebd_gate_host_supersite(L, n_max, U, J, Jnnn, K, jc, k, tau, _dptr(out)),
           "tebd_gate_host_supersite")
    return out.view(np.complex128).reshape(d ** 4, d ** 4)


class TEBD:
    """One simulation handle (see include/ptebd.h for every call's contract)."""

    def __init__(self, L, n_max, chi_max, U, J, Jnnn, K, jc, dt, w_cut=None, eps_rel=None, precision=None,
                 stream=None, u1=None):
        h = _c_void_p()
        _check(load().tebd_create(L, n_max, chi_max, U, J, Jnnn, K, jc, dt, ctypes.byref(h)), "tebd_create")
        self._h = h
        self.L, self.d, self.J = L, n_max + 1, J
        self.n_meas = L
        self._options(w_cut, eps_rel, precision, stream, u1)

    def _options(self, w_cut, eps_rel, precision, stream, u1):
        if w_cut is not None:
            self.set_option("w_cut", w_cut)
        if eps_rel is not None:
            self.set_option("eps_rel", eps_rel)
        if precision is not None:
            self.set_option("precision", precision)
        if u1 is not None:
            self.set_option("u1", 1 if u1 else 0)
        if stream is not None:
            self.set_stream(stream)

    def set_option(self, key: str, value: float):
        _check(load().tebd_set_option(self._h, key.encode(), float(value)), f"tebd_set_option({key})")

    def set_stream(self, stream_ptr: int):
        _check(load().tebd_set_stream(self._h, _c_void_p(stream_ptr)), "tebd_set_stream")

    def init_product(self, occ):
        occ = np.ascontiguousarray(occ, dtype=np.int32)
        _check(load().tebd_init_product(self._h, occ.ctypes.data_as(_P_int)), "tebd_init_product")

    def step(self, n: int = 1):
        _check(load().tebd_step(self._h, int(n)), "tebd_step")

    def layer(self, residue: int, full: bool):
        _check(load().tebd_layer(self._h, int(residue), int(bool(full))), "tebd_layer")

    def measure(self):
        n = np.empty(self.n_meas)
        cur = np.empty(self.n_meas - 1)
        _check(load().tebd_measure(self._h, _dptr(n), _dptr(cur)), "tebd_measure")
        return n, cur

    def stats(self):
        t, w = _c_double(), _c_double()
        chi = _c_int()
        _check(load().tebd_stats(self._h, ctypes.byref(t), ctypes.byref(w), ctypes.byref(chi)), "tebd_stats")
        return t.value, w.value, chi.value

    def device_bytes(self) -> float:
        out = _c_double()
        _check(load().tebd_device_bytes(self._h, ctypes.byref(out)), "tebd_device_bytes")
        return out.value

    def bond_dims(self):
        out = np.empty(self.L + 1, dtype=np.int32)
        _check(load().tebd_bond_dims(self._h, out.ctypes.data_as(_P_int)), "tebd_bond_dims")
        return out

    def get_site(self, k: int):
        chi = self.bond_dims()
        B = np.empty(2 * chi[k] * self.d * chi[k + 1])
        lam = np.empty(chi[k])
        _check(load().tebd_get_site(self._h, k, _dptr(B), _dptr(lam)), "tebd_get_site")
        return B.view(np.complex128).reshape(chi[k], self.d, chi[k + 1]), lam

    def get_lambda(self, k: int):
        chi = self.bond_dims()
        lam = np.empty(chi[k])
        _check(load().tebd_get_site(self._h, k, None, _dptr(lam)), "tebd_get_site")
        return lam

    def set_state(self, B, lam):
        chi = np.array([len(x) for x in lam], dtype=np.int32)
        Bs = [np.ascontiguousarray(b, dtype=np.complex128).view(np.float64).ravel() for b in B]
        ls = [np.ascontiguousarray(x, dtype=np.float64) for x in lam]
        Bp = (_P_double * len(Bs))(*[_dptr(b) for b in Bs])
        lp = (_P_double * len(ls))(*[_dptr(x) for x in ls])
        _check(load().tebd_set_state(self._h, chi.ctypes.data_as(_P_int), Bp, lp), "tebd_set_state")

    def set_charges(self, q):
        """Bond charge labels for the particle-number-blocked form (tebd_set_charges): q[k] holds, per
        Schmidt index of bond k, the boson count left of the bond, non-decreasing."""
        qs = [np.ascontiguousarray(x, dtype=np.int32) for x in q]
        qp = (_P_int * len(qs))(*[x.ctypes.data_as(_P_int) for x in qs])
        _check(load().tebd_set_charges(self._h, qp), "tebd_set_charges")

    def set_test_matrices(self, fn):
        """Source of the randomized truncation's Gaussian test matrices: fn(call, n, l) returns the
        n x l complex matrix of the call-th decomposition (an input of the method)."""
        def cb(call, n, l, out, _ctx):
            a = np.ascontiguousarray(fn(int(call), int(n), int(l)), dtype=np.complex128).reshape(n, l)
            ctypes.memmove(out, a.ctypes.data, a.nbytes)
        self._omega_cb = TEST_MATRIX_FN(cb) if fn is not None else TEST_MATRIX_FN()
        _check(load().tebd_set_test_matrices(self._h, self._omega_cb, None), "tebd_set_test_matrices")

    def get_charges(self, k: int):
        chi = self.bond_dims()
        out = np.empty(chi[k], dtype=np.int32)
        _check(load().tebd_get_charges(self._h, k, out.ctypes.data_as(_P_int)), "tebd_get_charges")
        return out

    def counters(self):
        g, k = ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().tebd_counters(self._h, ctypes.byref(g), ctypes.byref(k)), "tebd_counters")
        return g.value, k.value

    PROFILE_CLASSES = ("contract", "gram", "tridiag", "bisect", "eigvec", "project", "truncate", "measure")

    def graph_stats(self):
        """(accepted replays, replays undone, launches per replay) of option "graph"."""
        r, f, n = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().tebd_graph_stats(self._h, ctypes.byref(r), ctypes.byref(f), ctypes.byref(n)), "tebd_graph_stats")
        return r.value, f.value, n.value

    def profile(self):
        """{class: (ms, launches, work)} since profiling was (re)started."""
        out = {}
        for i, name in enumerate(self.PROFILE_CLASSES):
            ms, w = _c_double(), _c_double()
            n = ctypes.c_longlong()
            _check(load().tebd_profile(self._h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)),
                   "tebd_profile")
            out[name] = (ms.value, n.value, w.value)
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().tebd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SuperSiteTEBD(TEBD):
    """A handle of the super-site scheme (tebd_create_supersite): L physical sites as
    ceil(L / 2) super sites of local dimension (n_max + 1)^2.  L, d, get_site and
    bond_dims refer to the super sites; measure() returns the padded physical chain
    (2 ceil(L / 2) densities and one current fewer)."""

    def __init__(self, L, n_max, chi_max, U, J, Jnnn, K, jc, dt, w_cut=None, eps_rel=None, precision=None,
                 stream=None):
        h = _c_void_p()
        _check(load().tebd_create_supersite(L, n_max, chi_max, U, J, Jnnn, K, jc, dt, ctypes.byref(h)),
               "tebd_create_supersite")
        self._h = h
        self.L_phys = L
        self.L, self.d, self.J = (L + L % 2) // 2, (n_max + 1) ** 2, J
        self.n_meas = 2 * self.L
        self._options(w_cut, eps_rel, precision, stream, None)
