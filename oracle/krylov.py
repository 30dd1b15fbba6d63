"""FP64 oracle of the next basis builders: the Krylov-Hessenberg process and the
panel-blocked Hessenberg process.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

- Krylov-Hessenberg process (Sec. 4.1, Alg. 7): a basis of the Krylov space
  K_k(A, v) built Arnoldi-style, but each new vector A v_j is made zero at the
  pivot rows of the earlier vectors (the preselected vectors z_i are unit
  vectors at those rows) instead of orthogonal to them, and scaled so that its
  largest-magnitude entry (its pivot) is 1.  The coefficients form the upper
  Hessenberg matrix of the relation A v_j = sum_{i <= j} h_ij v_i + h_{j+1,j} v_{j+1}.
- Blocked Hessenberg process (the level-3 form of Alg. 8 that Table 1's "Block"
  row and the closing future-work passage point to): columns are processed in
  panels of r; a panel is factored by the unblocked steps restricted to its
  columns, then the trailing columns take the whole panel at once (solve with
  the panel's unit lower triangle at its pivot rows, then one rank-r update).
  In exact arithmetic it returns what Alg. 8 returns.
"""
from __future__ import annotations

import numpy as np

__all__ = ["krylov_hessenberg", "hessenberg_blocked", "solve_krylov_eig"]


def krylov_hessenberg(Amul, v, k: int):
    """Alg. 7: returns (V n x k, Hbar k x (k-1), pivots).  Amul(x) applies A to a
    vector.  Pivot = first index of the largest magnitude (as LAPACK's i?amax)."""
    v = np.asarray(v, dtype=np.float64).copy()
    n = v.shape[0]
    V = np.zeros((n, k))
    H = np.zeros((k, max(k - 1, 0)))
    piv = np.zeros(k, dtype=np.int64)
    r = int(np.argmax(np.abs(v)))
    V[:, 0] = v / v[r]
    piv[0] = r
    for j in range(k - 1):
        w = np.asarray(Amul(V[:, j]), dtype=np.float64).copy()
        for i in range(j + 1):
            c = w[piv[i]]                 # coefficient read from the current vector
            H[i, j] = c
            w = w - c * V[:, i]
        r = int(np.argmax(np.abs(w)))
        H[j + 1, j] = w[r]
        V[:, j + 1] = w / w[r]
        piv[j + 1] = r
    return V, H, piv


def hessenberg_blocked(W, r: int):
    """Panel-blocked Hessenberg process on W (n x k, full column rank assumed):
    returns (Q, pivots) with Q = P^T L of row-pivoted LU, as Alg. 8."""
    Q = np.array(W, dtype=np.float64, order="F", copy=True)
    n, k = Q.shape
    piv = np.zeros(k, dtype=np.int64)
    for c0 in range(0, k, r):
        c1 = min(k, c0 + r)
        # panel: the unblocked steps on columns c0 .. c1-1 only
        for j in range(c0, c1):
            q = Q[:, j]
            p = int(np.argmax(np.abs(q)))
            Q[:, j] = q / q[p]
            piv[j] = p
            w = Q[p, j + 1:c1].copy()
            if w.size:
                Q[:, j + 1:c1] -= np.outer(Q[:, j], w)
        if c1 < k:
            # trailing columns: T <- T - L_panel (L11^-1 T[pivot rows]); L11 is the
            # panel's unit lower triangle at its pivot rows
            L = Q[:, c0:c1]
            L11 = L[piv[c0:c1], :]
            U12 = np.linalg.solve(L11, Q[piv[c0:c1], c1:])
            Q[:, c1:] -= L @ U12
    return Q, piv


def solve_krylov_eig(A_mul, v0, m: int, restarts: int, k: int):
    """Krylov-Hessenberg basis with OFRR for a symmetric operator (Sec. 4.1,
    Alg. 7 for the basis, Alg. 3 for the projection; the sparse experiment of
    Sec. 5.2.2): `restarts + 1` cycles, each building the m-dimensional basis
    of K_m(A, v) by Alg. 7 and solving the projected pencil
    (V^T A V) y = theta (V^T V) y; the next cycle restarts from the single Ritz
    vector of the largest Ritz value.  Returns (theta: the k largest Ritz
    values, descending; X: their unit Ritz vectors; res: relative residuals
    |A x - theta x| / |theta|)."""
    from .ofrr import pencil_eig, residual_eig
    v = np.asarray(v0, dtype=np.float64)
    for _ in range(restarts + 1):
        V, _, _ = krylov_hessenberg(A_mul, v, m)
        AV = np.asarray(A_mul(V), dtype=np.float64)
        theta, Y = pencil_eig(V.T @ AV, V.T @ V)
        order = np.argsort(-theta)
        theta, Y = theta[order], Y[:, order]
        X = V @ Y
        X = X / np.linalg.norm(X, axis=0)
        v = X[:, 0]
    return theta[:k], X[:, :k], residual_eig(A_mul, X[:, :k], theta[:k])
