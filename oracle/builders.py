"""FP64 oracle of the basis builders the paper compares with the Hessenberg
process (Sec. 4, Table 1; Table 3's timings).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each takes an n x k block W and returns its basis Q (and the triangular
factor R of W = Q R for the Gram-Schmidt methods, or the pivot rows for the
Hessenberg process), column by column as the method's name says:

- MGS-L: column j is reduced against the earlier basis vectors one at a time,
  each coefficient the dot product with the column as it stands (modified
  Gram-Schmidt, left-looking), then normalised;
- MGS-R: once column j is normalised it is removed from every later column
  (right-looking);
- CGS: all coefficients of column j from the column as it came in (classical),
  removed together; CGS-2 repeats that once (re-orthogonalisation);
- Hess-L: column j takes the eliminations of all earlier columns when it is
  reached (coefficients read at their pivot rows), then its pivot is its
  largest-magnitude entry (first index on ties) and it is scaled to 1 there.
"""
from __future__ import annotations

import numpy as np

__all__ = ["mgs_left", "mgs_right", "cgs", "cgs2", "hess_left"]


def mgs_left(W):
    Q = np.array(W, dtype=np.float64, order="F", copy=True)
    n, k = Q.shape
    R = np.zeros((k, k))
    for j in range(k):
        for i in range(j):
            R[i, j] = Q[:, i] @ Q[:, j]
            Q[:, j] = Q[:, j] - R[i, j] * Q[:, i]
        R[j, j] = np.linalg.norm(Q[:, j])
        Q[:, j] = Q[:, j] / R[j, j]
    return Q, R


def mgs_right(W):
    Q = np.array(W, dtype=np.float64, order="F", copy=True)
    n, k = Q.shape
    R = np.zeros((k, k))
    for j in range(k):
        R[j, j] = np.linalg.norm(Q[:, j])
        Q[:, j] = Q[:, j] / R[j, j]
        for c in range(j + 1, k):
            R[j, c] = Q[:, j] @ Q[:, c]
            Q[:, c] = Q[:, c] - R[j, c] * Q[:, j]
    return Q, R


def _cgs(W, passes):
    Q = np.array(W, dtype=np.float64, order="F", copy=True)
    n, k = Q.shape
    R = np.zeros((k, k))
    for j in range(k):
        for _ in range(passes if j > 0 else 0):
            r = Q[:, :j].T @ Q[:, j]
            Q[:, j] = Q[:, j] - Q[:, :j] @ r
            R[:j, j] += r
        R[j, j] = np.linalg.norm(Q[:, j])
        Q[:, j] = Q[:, j] / R[j, j]
    return Q, R


def cgs(W):
    return _cgs(W, 1)


def cgs2(W):
    return _cgs(W, 2)


def hess_left(W):
    Q = np.array(W, dtype=np.float64, order="F", copy=True)
    n, k = Q.shape
    piv = np.zeros(k, dtype=np.int64)
    for j in range(k):
        w = Q[:, j].copy()
        for i in range(j):
            w = w - w[piv[i]] * Q[:, i]
        p = int(np.argmax(np.abs(w)))
        Q[:, j] = w / w[p]
        piv[j] = p
    return Q, piv
