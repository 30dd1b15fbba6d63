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


def _lanczos_full(A, v, m):
    """An orthonormal basis of K_m(A, v): Arnoldi with two passes of modified
    Gram-Schmidt per vector (an independent construction of the same space)."""
    n = v.shape[0]
    Q = np.zeros((n, m))
    Q[:, 0] = v / np.linalg.norm(v)
    for j in range(1, m):
        w = A @ Q[:, j - 1]
        for _ in range(2):
            for i in range(j):
                w = w - (Q[:, i] @ w) * Q[:, i]
        Q[:, j] = w / np.linalg.norm(w)
    return Q


def test_solve_krylov_eig_equals_classical_rr_on_the_krylov_space():
    """One cycle of Alg. 7 + Alg. 3 gives the Ritz values of K_m(A, v) (OFRR
    equals classical RR on the same span, Sec. 3); with restarts every cycle
    starts from the top Ritz vector of the previous one."""
    import workloads as wl
    rp, ci, va, _ = wl.grid_schrodinger_csr(11, 10.0, 5300)
    Amul = O.csr_apply(rp, ci, va)
    A = Amul(np.eye(121))
    v = wl.uniform_block(121, 1, 5301)[:, 0]
    th, X, res = K.solve_krylov_eig(Amul, v, 20, 0, 6)
    Q = _lanczos_full(A, v, 20)
    ref = np.sort(np.linalg.eigvalsh(Q.T @ A @ Q))[::-1][:6]
    assert np.allclose(th, ref, rtol=1e-10, atol=0)
    assert np.allclose(res, O.residual_eig(Amul, X, th), rtol=1e-12)
    # two restarts, composed by hand with the orthonormal construction
    th2, X2, _ = K.solve_krylov_eig(Amul, v, 20, 2, 6)
    w = v
    for _ in range(3):
        Q = _lanczos_full(A, w, 20)
        lam, Z = np.linalg.eigh(Q.T @ A @ Q)
        w = Q @ Z[:, -1]
    assert np.allclose(th2, lam[::-1][:6], rtol=1e-9, atol=0)
    # the largest eigenvalue of the grid operator is reached
    assert abs(th2[0] - np.linalg.eigvalsh(A)[-1]) < 1e-8 * th2[0]
