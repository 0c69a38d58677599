"""The two Gram routes the GPU path uses for a charge block (reading U4), checked in
plain numpy FP64 against LAPACK's SVD: for a block M (b x n) with a decaying spectrum,
  left  (b <= n): eigenvectors u_k of M M^+, s_k = |u_k^+ M|, V^+ rows u_k^+ M / s_k;
  right (n <  b): eigenvectors z_k of M^+ M, s_k = |M z_k|,   V^+ rows z_k^+;
both give the singular values to rounding (second order in the eigenvector error) and
the same right singular subspaces.  This pins the reading the kernels implement; it
calls no GPU code."""
import numpy as np
import pytest


def _block(rng, b, n, decay):
    k = min(b, n)
    U, _ = np.linalg.qr(rng.standard_normal((b, k)) + 1j * rng.standard_normal((b, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    s = np.exp(-decay * np.arange(k) / k)
    s /= np.linalg.norm(s)
    return (U * s) @ V.conj().T


def _left(M):
    w, U = np.linalg.eigh(M @ M.conj().T)
    U = U[:, ::-1][:, :min(M.shape)]
    Y = U.conj().T @ M
    s = np.linalg.norm(Y, axis=1)
    return s, Y / s[:, None]


def _right(M):
    w, Z = np.linalg.eigh(M.conj().T @ M)
    Z = Z[:, ::-1]
    s = np.linalg.norm(M @ Z, axis=0)
    return s, Z.conj().T


@pytest.mark.parametrize("b,n", [(200, 50), (300, 30), (90, 60)])
def test_both_routes_match_the_svd(b, n):
    rng = np.random.default_rng(240105301)
    M = _block(rng, b, n, decay=10.0)  # smallest singular value ~ 4e-5 of the largest
    _, sv, Vh = np.linalg.svd(M, full_matrices=False)
    for route in (_left, _right):
        s, Wh = route(M)
        order = np.argsort(-s)
        s, Wh = s[order], Wh[order]
        assert np.max(np.abs(s - sv)) < 1e-14
        # each kept row spans the same right singular direction (up to a phase)
        overlap = np.abs(np.sum(Wh.conj() * Vh, axis=1))
        assert np.max(np.abs(overlap - 1.0)) < 1e-10

