"""Pins of the comparator basis builders' oracle (CPU only): the Gram-Schmidt
variants give the QR factorisation (Q orthonormal, R upper triangular with a
positive diagonal, W = Q R), equal to LAPACK's Householder QR with its signs
fixed; left- and right-looking MGS and CGS-2 agree; the left-looking
Hessenberg process gives Algorithm 8's pivots and basis (row-pivoted LU)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import builders as B
from oracle import ofrr as O


def _block(n, k, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, (n, k))   # Table 3's U(0,1) blocks


@pytest.mark.parametrize("fn", [B.mgs_left, B.mgs_right, B.cgs, B.cgs2])
def test_gram_schmidt_is_the_qr_factorisation(fn):
    W = _block(300, 20, 1)
    Q, R = fn(W)
    assert np.abs(Q @ R - W).max() < 1e-13 * np.abs(W).max()
    assert np.allclose(np.tril(R, -1), 0.0) and np.all(np.diag(R) > 0)
    Qh, Rh = np.linalg.qr(W)
    sgn = np.sign(np.diag(Rh))
    assert np.abs(Q - Qh * sgn).max() < 1e-10
    assert np.abs(R - Rh * sgn[:, None]).max() < 1e-10 * np.abs(Rh).max()


def test_orthogonality_ordering_on_an_ill_conditioned_block():
    """Loss of orthogonality: CGS-2 ~ u, MGS ~ u cond(W), CGS ~ u cond(W)^2
    (the stability column of Table 1), on a block with cond ~ 1e6."""
    rng = np.random.default_rng(2)
    U, _ = np.linalg.qr(rng.standard_normal((400, 30)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    W = (U * np.logspace(0, -6, 30)) @ V.T
    loss = {f.__name__: np.abs(f(W)[0].T @ f(W)[0] - np.eye(30)).max() for f in (B.cgs, B.mgs_left, B.cgs2)}
    assert loss["cgs2"] < 1e-14 < loss["mgs_left"] < 1e-8 < loss["cgs"]
    Qr, _ = B.mgs_right(W)
    assert np.abs(Qr - B.mgs_left(W)[0]).max() < 1e-8


def test_hess_left_is_algorithm_8():
    W = _block(500, 24, 3)
    Q, piv = B.hess_left(W)
    Qo, pivo, keep, _ = O.hessenberg(W)
    assert keep.all() and np.array_equal(piv, pivo)
    assert np.abs(Q - Qo).max() < 1e-12
    P, L, U = sla.lu(W)
    assert np.abs(Q - P @ L).max() < 1e-12
