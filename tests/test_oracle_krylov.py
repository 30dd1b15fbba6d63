"""Pins of the next basis builders' oracle (CPU only): the Krylov-Hessenberg
process against Alg. 8 applied to the explicit Krylov matrix, its Hessenberg
relation and pivot structure, exact eigenvalues at full dimension; the blocked
Hessenberg process against the unblocked one and against row-pivoted LU."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import krylov as K
from oracle import ofrr as O


def _sym(n, seed, lo=1.0, hi=2.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(lo, hi, n)
    return (Q * lam) @ Q.T, lam


def test_krylov_hessenberg_equals_hessenberg_of_krylov_matrix():
    """The j-th vector is the unique vector of K_j zero at the earlier pivot rows
    with unit pivot: Alg. 7 equals Alg. 8 (row-pivoted LU) of [v, Av, ..., A^(k-1) v]."""
    A, _ = _sym(80, 1)
    v = np.random.default_rng(2).uniform(0, 1, 80)
    k = 7
    V, H, piv = K.krylov_hessenberg(lambda x: A @ x, v, k)
    Kr = np.empty((80, k))
    Kr[:, 0] = v
    for j in range(1, k):
        Kr[:, j] = A @ Kr[:, j - 1]
    Q, p8, keep, _ = O.hessenberg(Kr)
    assert keep.all() and np.array_equal(piv, p8)
    assert np.abs(V - Q).max() < 1e-8


def test_krylov_hessenberg_relation_and_structure():
    A, _ = _sym(120, 3, -1.0, 3.0)
    v = np.random.default_rng(4).standard_normal(120)
    k = 12
    V, H, piv = K.krylov_hessenberg(lambda x: A @ x, v, k)
    # A V_(k-1) = V_k Hbar, Hbar upper Hessenberg
    assert np.abs(A @ V[:, :k - 1] - V @ H).max() < 1e-12 * np.abs(A).sum(axis=1).max() * 10
    assert np.all(np.tril(H, -2) == 0)
    # unit pivot, |V| <= 1, exact zeros of later vectors at earlier pivot rows
    assert np.all(V[piv, np.arange(k)] == 1.0) and np.abs(V).max() <= 1.0
    for j in range(k):
        assert np.all(V[piv[:j], j] == 0.0)
    assert len(set(piv.tolist())) == k


def test_krylov_hessenberg_full_dimension_gives_exact_eigenvalues():
    """With k = n the basis spans the space: the orthogonalization-free
    Rayleigh-Ritz over it (Alg. 3) returns the eigenvalues of A."""
    A, lam = _sym(10, 5)
    V, H, piv = K.krylov_hessenberg(lambda x: A @ x, np.ones(10), 10)
    th = sla.eigh(V.T @ A @ V, V.T @ V, eigvals_only=True)
    assert np.abs(np.sort(th) - lam).max() < 1e-8


@pytest.mark.parametrize("r", [1, 3, 8, 24])
def test_blocked_hessenberg_equals_unblocked_and_lu(r):
    W = np.random.default_rng(6).uniform(0, 1, (200, 24))
    Q, piv = K.hessenberg_blocked(W, r)
    Q8, p8, keep, _ = O.hessenberg(W)
    assert keep.all() and np.array_equal(piv, p8)
    if r == 1:
        assert np.array_equal(Q, Q8)          # the same operations in the same order
    else:
        assert np.abs(Q - Q8).max() < 1e-12
    P, L, U = sla.lu(W)
    assert np.abs(Q - P @ L).max() < 1e-12
