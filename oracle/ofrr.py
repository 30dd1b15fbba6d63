"""FP64 oracle: subspace iteration + Hessenberg basis + orthogonalization-free RR.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: "Mixed Precision Orthogonalization-Free Projection Methods for
Eigenvalue and Singular Value Problems" (arXiv 2505.00281).  Each function
names the passage it follows.  Readings of passages that are silent, garbled
or ambiguous are marked READING.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

__all__ = [
    "round_bf16", "round_e4m3", "e4m3_decode", "e4m3_scale_exp", "quantize_e4m3", "colscale_inf", "hessenberg", "hessenberg_tol",
    "gram", "dense_apply", "csr_apply", "csr_gershgorin",
    "pencil_eig", "pencil_svd", "rayleigh_ritz_eig", "rayleigh_ritz_svd",
    "chebyshev_filter", "residual_eig", "residual_svd",
    "solve_eig", "solve_svd", "SolveResult", "svd_correction_sweep",
]

EPS64 = 2.0 ** -52
EPS32 = 2.0 ** -23
EPSBF16 = 2.0 ** -7


# --------------------------------------------------------------------------
# rounding to the storage formats the GPU path uses (for building the exact
# operands a kernel sees; the oracle itself computes in FP64)
# --------------------------------------------------------------------------
def round_bf16(x) -> np.ndarray:
    """Round to bfloat16 (round-to-nearest-even on the FP32 bit pattern), return FP64.

    x is first rounded to FP32 (RNE), then the low 16 bits are rounded away.
    NaN/Inf are not expected in inputs and are not special-cased.
    """
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(x))


E4M3_MAX = 448.0


def e4m3_decode(code) -> np.ndarray:
    """Value of an FP8-E4M3 byte (OCP 8-bit float, 'fn' variant): sign bit, 4
    exponent bits (bias 7), 3 mantissa bits; exponent 0 is subnormal (m/8 2^-6);
    S.1111.111 is NaN, there is no infinity.  FP64 output."""
    c = np.asarray(code, dtype=np.int64)
    sgn = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = (c & 7).astype(np.float64)
    val = np.where(e == 0, m / 8.0 * 2.0 ** -6, (1.0 + m / 8.0) * np.exp2(e.astype(np.float64) - 7.0))
    val = np.where((c & 0x7F) == 0x7F, np.nan, val)
    return sgn * val


def round_e4m3(x) -> np.ndarray:
    """Round to FP8-E4M3 as the FP8 path does (READING: the GPU converts FP64 to
    FP32 first, so both sides take the same two steps): FP32 round-to-nearest-even,
    then to the nearest E4M3 value, ties to even mantissa, saturating at +-448.
    The spacing is 2^(E-3) for |f| in [2^E, 2^(E+1)), E >= -6, and 2^-9 below 2^-6."""
    f = np.asarray(np.asarray(x, dtype=np.float32), dtype=np.float64)
    a = np.abs(f)
    E = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    q = np.exp2(np.maximum(E, -6.0) - 3.0)
    r = np.rint(f / q) * q                       # f / q is exact (q a power of two)
    return np.clip(r, -E4M3_MAX, E4M3_MAX)


def e4m3_scale_exp(m):
    """Largest e with m 2^e <= 448, clamped to [-126, 126]; 0 where m = 0."""
    m = np.asarray(m, dtype=np.float64)
    fr, ex = np.frexp(np.where(m > 0, m, 1.0))     # m = fr 2^ex, fr in [0.5, 1)
    e = 8 - (ex - 1) - (2.0 * fr > 1.75)
    e = np.clip(e, -126, 126)
    return np.where(m > 0, e, 0).astype(np.int64)


def quantize_e4m3(X, by_rows: bool):
    """E4M3 values of X with one power-of-two scale per column (or per row):
    returns (values of the E4M3 codes, FP64, same shape as X; inverse scales 2^-e)."""
    X = np.asarray(X, dtype=np.float64)
    m = np.max(np.abs(X), axis=1 if by_rows else 0) if X.size else np.zeros(0)
    e = e4m3_scale_exp(m)
    s = np.exp2(e.astype(np.float64))
    Xs = X * (s[:, None] if by_rows else s[None, :])
    return round_e4m3(Xs), np.exp2(-e.astype(np.float64))


# --------------------------------------------------------------------------
# Sec. 2 (column scaling after each product) and Sec. 4.1 (inf-norm scaling)
# --------------------------------------------------------------------------
def colscale_inf(X: np.ndarray) -> np.ndarray:
    """Scale every column to unit infinity norm (Sec. 2, column scaling; Sec. 4.1.2).

    Zero columns are left at zero.
    """
    X = np.asarray(X, dtype=np.float64)
    m = np.max(np.abs(X), axis=0) if X.shape[0] else np.zeros(X.shape[1])
    m = np.where(m > 0, m, 1.0)
    return np.asfortranarray(X / m)


# --------------------------------------------------------------------------
# Algorithm 8: Hessenberg process for a block, right-looking
# --------------------------------------------------------------------------
def hessenberg_tol(arith: str, k: int) -> float:
    """Column-skip tolerance (Sec. 5.2: set relative to the machine epsilon of
    the arithmetic).  READING: 4 k eps, with eps that of the arithmetic that
    runs the process (FP64 2^-52, FP32 2^-23) and k the block width, applied
    relative to the column's infinity norm on entry (equivalent to
    inf-normalising the columns first, Sec. 2).  The factor 4k covers the
    rounding residue that k eliminations leave in an exactly dependent column
    (plain eps keeps such columns as rounding noise)."""
    return 4.0 * max(k, 1) * {"f64": EPS64, "f32": EPS32}[arith]


def hessenberg(W: np.ndarray, tol: float | None = None, arith: str = "f64"):
    """Right-looking Hessenberg process, Algorithm 8 (Sec. 4.2.2).

    For j = 1..k: r = argmax_i |Q_ij| (READING: the first index among equal
    magnitudes, as LAPACK's i?amax); if |Q_rj| is at least tol times the
    column's entry infinity norm, scale the column by 1/Q_rj, record pi_j = r
    and, for every later column i, subtract Q_ri times the scaled column
    (READING of the garbled subscripts: the weight is the entry of column i
    in the pivot row r of the current column); otherwise mark the column as
    skipped.  Skipped columns are removed at the end.

    ``arith`` is "f64" (the definition) or "f32": the same steps in IEEE FP32
    with separately rounded multiply and subtract, which is what the GPU
    kernel executes, so that both sides take every argmax decision in the same
    precision.

    Returns (Q compacted to the kept columns, pivots pi (int, -1 for skipped),
    keep mask, Q_full with skipped columns set to zero).
    """
    dt = np.float64 if arith == "f64" else np.float32
    Q = np.array(W, dtype=dt, order="F", copy=True)
    n, k = Q.shape
    if tol is None:
        tol = hessenberg_tol(arith, k)
    colmax = np.max(np.abs(Q), axis=0) if n else np.zeros(k, dt)
    thr = (dt(tol) * colmax).astype(dt)
    keep = np.ones(k, dtype=bool)
    piv = np.full(k, -1, dtype=np.int64)
    for j in range(k):
        q = Q[:, j]
        if n == 0:
            keep[j] = False
            continue
        r = int(np.argmax(np.abs(q)))
        if np.abs(q[r]) >= thr[j] and q[r] != 0:
            q = (q / q[r]).astype(dt)
            Q[:, j] = q
            piv[j] = r
            w = Q[r, j + 1:].copy()          # weights read before the update
            if w.size:
                Q[:, j + 1:] = (Q[:, j + 1:] - np.outer(q, w).astype(dt)).astype(dt)
        else:
            keep[j] = False
            Q[:, j] = 0
    Qfull = Q
    return np.asfortranarray(Qfull[:, keep]), piv, keep, Qfull


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
def dense_apply(A: np.ndarray):
    """Return (X -> A X, X -> A^T X) for a dense FP64 matrix."""
    A = np.asarray(A, dtype=np.float64)
    return (lambda X: A @ X), (lambda X: A.T @ X)


def csr_apply(row_ptr, col_idx, values, ncols: int | None = None):
    """Return X -> A X for a CSR matrix (values promoted to FP64)."""
    import scipy.sparse as sp

    n = len(row_ptr) - 1
    ncols = n if ncols is None else ncols
    M = sp.csr_matrix((np.asarray(values, np.float64), np.asarray(col_idx), np.asarray(row_ptr)),
                      shape=(n, ncols))
    return lambda X: M @ X


def csr_gershgorin(row_ptr, col_idx, values):
    """Gershgorin lower and upper bounds of a symmetric CSR matrix (FP64)."""
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col_idx, np.int64)
    va = np.asarray(values, np.float64)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    d = np.zeros(len(rp) - 1)
    off = np.zeros(len(rp) - 1)
    isd = rows == ci
    np.add.at(d, rows[isd], va[isd])
    np.add.at(off, rows[~isd], np.abs(va[~isd]))
    return float(np.min(d - off)), float(np.max(d + off))


def gram(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """X^T Y in FP64 (the projection products of Algorithms 3 and 5)."""
    return np.asarray(X, np.float64).T @ np.asarray(Y, np.float64)


# --------------------------------------------------------------------------
# small projected problems
# --------------------------------------------------------------------------
def _whitener(G: np.ndarray):
    """Return (W, rank) with W^T G W = I on the numerically nonsingular part.

    Cholesky when G is numerically positive definite; otherwise (READING of
    the breakdown case, which the paper leaves open) the FP64 eigenvectors
    of G scaled by 1/sqrt(eigenvalue), keeping eigenvalues above
    u64 * lambda_max(G).
    """
    G = 0.5 * (G + G.T)
    try:
        L = np.linalg.cholesky(G)
        if np.min(np.diag(L)) ** 2 > 64 * EPS64 * np.max(np.diag(G)):
            W = sla.solve_triangular(L, np.eye(G.shape[0]), lower=True).T
            return W, G.shape[0]
    except np.linalg.LinAlgError:
        pass
    lam, E = np.linalg.eigh(G)
    ok = lam > EPS64 * max(lam[-1], 0.0) * G.shape[0]
    W = E[:, ok] / np.sqrt(lam[ok])
    return W, int(ok.sum())


def pencil_eig(H: np.ndarray, G: np.ndarray):
    """Solve H Y = G Y Theta (the generalized eigenproblem B Y = M Y Lambda of Algorithm 3), FP64.

    H symmetric, G symmetric positive (semi)definite.  Returns theta ascending
    and Y with Y^T G Y = I.  When G is numerically definite this is LAPACK's
    symmetric-definite generalized eigensolver; otherwise the pencil is
    restricted to the range of G (see ``_whitener``).
    """
    H = 0.5 * (H + H.T)
    G = 0.5 * (G + G.T)
    W, r = _whitener(G)
    if r == G.shape[0]:
        theta, Y = sla.eigh(H, G)
        return theta, Y
    C = W.T @ H @ W
    theta, Z = np.linalg.eigh(0.5 * (C + C.T))
    return theta, W @ Z


def pencil_svd(B: np.ndarray, Gu: np.ndarray, Gv: np.ndarray):
    """The 2-by-2 block pencil of Eq. (gev for svd matrix), Algorithm 5.

    Solves [[0, B], [B^T, 0]] [y; z] = s [[Gu, 0], [0, Gv]] [y; z] literally
    (dimension k1 + k2), keeps the min(k1, k2) largest eigenvalues (the
    positive ones; Sec. 3.2: the spectrum is +-s plus zeros) and returns
    (s descending, Y, Z) with the pencil normalisation
    [y; z]^T diag(Gu, Gv) [y; z] = 1.  The sqrt(2) lift of the theorem in
    Sec. 3.2 is applied by the caller.
    """
    k1, k2 = B.shape
    K = np.zeros((k1 + k2, k1 + k2))
    K[:k1, k1:] = B
    K[k1:, :k1] = B.T
    M = np.zeros_like(K)
    M[:k1, :k1] = Gu
    M[k1:, k1:] = Gv
    w, E = pencil_eig(K, M)
    r = min(k1, k2)
    order = np.argsort(-w)[:r]
    return w[order], E[:k1, order], E[k1:, order]


def rayleigh_ritz_eig(A_mul, U: np.ndarray):
    """Algorithm 3 (OFRR for eigenvalue problems): B = U^T A U, M = U^T U,
    B Y = M Y Lambda, U~ = U Y.  Returns (theta ascending, Y, U~, AU)."""
    AU = A_mul(U)
    B = U.T @ AU
    M = U.T @ U
    theta, Y = pencil_eig(B, M)
    return theta, Y, U @ Y, AU


def rayleigh_ritz_svd(A_mul, U: np.ndarray, V: np.ndarray):
    """Algorithm 5 (OFRR for the SVD): solve the block pencil for its positive
    eigenvalues and lift with sqrt(2) U Y, sqrt(2) V Z (theorem of Sec. 3.2).
    Returns (s descending, U~, V~, Y, Z)."""
    AV = A_mul(V)
    B = U.T @ AV
    s, Y, Z = pencil_svd(B, U.T @ U, V.T @ V)
    return s, math.sqrt(2.0) * (U @ Y), math.sqrt(2.0) * (V @ Z), Y, Z


# --------------------------------------------------------------------------
# scaled Chebyshev filter (the "chebfsi" family the paper cites in Sec. 2)
# --------------------------------------------------------------------------
def chebyshev_filter(A_mul, X: np.ndarray, degree: int, a: float, b_up: float, a0: float):
    """Degree-d scaled Chebyshev filter damping [a, b_up] and normalised at a0.

    e = (b_up - a)/2, c = (b_up + a)/2, s1 = e/(a0 - c);
    Y1 = (s1/e)(A - cI)X;  s_{j+1} = 1/(2/s1 - s_j);
    Y_{j+1} = (2 s_{j+1}/e)(A - cI)Y_j - s_j s_{j+1} Y_{j-1}.
    The result equals T_d((A - cI)/e) X / T_d((a0 - c)/e).
    """
    e = (b_up - a) / 2.0
    c = (b_up + a) / 2.0
    s1 = e / (a0 - c)
    Y0 = np.asarray(X, np.float64)
    Y1 = (s1 / e) * (A_mul(Y0) - c * Y0)
    s = s1
    for _ in range(2, degree + 1):
        sn = 1.0 / (2.0 / s1 - s)
        Y2 = (2.0 * sn / e) * (A_mul(Y1) - c * Y1) - (s * sn) * Y0
        Y0, Y1, s = Y1, Y2, sn
    return Y1


# --------------------------------------------------------------------------
# residuals (Sec. 5.2.2: ||A v - lambda v||_2 / |lambda| with ||v||_2 = 1)
# --------------------------------------------------------------------------
def residual_eig(A_mul, X: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Relative residual ||A x - theta x|| / |theta| per column, x normalised."""
    X = np.asarray(X, np.float64)
    nrm = np.linalg.norm(X, axis=0)
    Xn = X / np.where(nrm > 0, nrm, 1.0)
    R = A_mul(Xn) - Xn * theta
    return np.linalg.norm(R, axis=0) / np.abs(theta)


def residual_svd(A_mul, At_mul, U, V, s) -> np.ndarray:
    """READING for the SVD residual (the paper prints none):
    sqrt(||A v - s u||^2 + ||A^T u - s v||^2) / s with unit u and v."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    Un = U / np.linalg.norm(U, axis=0)
    Vn = V / np.linalg.norm(V, axis=0)
    r1 = np.linalg.norm(A_mul(Vn) - Un * s, axis=0)
    r2 = np.linalg.norm(At_mul(Un) - Vn * s, axis=0)
    return np.sqrt(r1 ** 2 + r2 ** 2) / s


# --------------------------------------------------------------------------
# Algorithm 1 coupled with Algorithm 3 / 5 (the RR output replaces the QR
# output as the next start block, Sec. 2) with Algorithm 8 as the basis step
# --------------------------------------------------------------------------
@dataclass
class SolveResult:
    values: np.ndarray            # k wanted Ritz values / singular values
    X: np.ndarray                 # eigenvectors (or right singular vectors V~)
    U: np.ndarray | None          # left singular vectors (SVD only)
    res: np.ndarray               # residuals of the k wanted pairs
    sweeps: int
    n_converged: int
    history: list = field(default_factory=list)   # per sweep: (values, res)


def _basis(W, hess: bool):
    if hess:
        return hessenberg(W, arith="f64")[0]
    return colscale_inf(W)


def solve_eig(A_mul, n: int, k: int, V0: np.ndarray, *, which: str = "largest",
              filter: str = "power", degree: int = 1, max_sweeps: int = 50,
              tol: float = 1e-10, hess: bool = True, bounds=None) -> SolveResult:
    """Subspace iteration with OFRR (Algorithms 1, 3, 8) in FP64.

    Per sweep: the filter (``degree`` products with A, each followed by the
    basis step, or a degree-d scaled Chebyshev filter followed by the basis
    step), then OFRR over the filtered block, then the residual check of the
    k wanted pairs.  The Ritz vectors start the next sweep.  ``bounds`` =
    (lower, upper) spectral bounds for the Chebyshev filter (Gershgorin).
    READING for the Chebyshev interval (not in the paper): first sweep damps
    [lo + 0.1 (up - lo), up] normalised at lo; later sweeps damp
    [max Ritz value, up] normalised at the min Ritz value.
    """
    V = colscale_inf(V0)
    hist = []
    theta_all = None
    res = None
    X = None
    for sweep in range(1, max_sweeps + 1):
        if filter == "power":
            for _ in range(degree):
                V = _basis(A_mul(V), hess)
        elif filter == "chebyshev":
            lo, up = bounds
            if theta_all is None:
                a, a0 = lo + 0.1 * (up - lo), lo
            else:
                a, a0 = float(np.max(theta_all)), float(np.min(theta_all))
            V = _basis(chebyshev_filter(A_mul, V, degree, a, up, a0), hess)
        else:
            raise ValueError(filter)
        theta, Y, X, _ = rayleigh_ritz_eig(A_mul, V)
        order = np.argsort(-theta) if which == "largest" else np.argsort(theta)
        theta_all = theta[order]
        X = X[:, order]
        X = X / np.linalg.norm(X, axis=0)
        res = residual_eig(A_mul, X[:, :k], theta_all[:k])
        hist.append((theta_all[:k].copy(), res.copy()))
        nconv = int(np.sum(res <= tol))
        if nconv >= k:
            return SolveResult(theta_all[:k], X[:, :k], None, res, sweep, nconv, hist)
        V = X
    return SolveResult(theta_all[:k], X[:, :k], None, res, max_sweeps,
                       int(np.sum(res <= tol)), hist)


def solve_svd(A_mul, At_mul, m: int, n: int, k: int, V0: np.ndarray, *,
              degree: int = 1, max_sweeps: int = 50, tol: float = 1e-10,
              hess: bool = True) -> SolveResult:
    """Subspace iteration for the largest singular triplets with OFRR for the
    SVD (Algorithms 1, 5, 8; Sec. 4: the SVD adds the products with A^T).

    Per sweep: ``degree`` times U = basis(A V), V = basis(A^T U); then
    Algorithm 5 on (U, V); the right Ritz vectors start the next sweep.
    """
    V = colscale_inf(V0)
    hist = []
    for sweep in range(1, max_sweeps + 1):
        for _ in range(degree):
            U = _basis(A_mul(V), hess)
            V = _basis(At_mul(U), hess)
        s, Ut, Vt, _, _ = rayleigh_ritz_svd(A_mul, U, V)
        res = residual_svd(A_mul, At_mul, Ut[:, :k], Vt[:, :k], s[:k])
        hist.append((s[:k].copy(), res.copy()))
        nconv = int(np.sum(res <= tol))
        if nconv >= k:
            return SolveResult(s[:k], Vt[:, :k], Ut[:, :k], res, sweep, nconv, hist)
        V = Vt
    return SolveResult(s[:k], Vt[:, :k], Ut[:, :k], res, max_sweeps,
                       int(np.sum(res <= tol)), hist)


# --------------------------------------------------------------------------
# refinement of the SVD in FP64 (not in the paper: the paper's method stops at
# the basis precision, Sec. 2; this is the correction sweep the GPU path runs
# in FP64-accurate arithmetic when its low-precision corrections stall)
# --------------------------------------------------------------------------
def svd_correction_sweep(A_mul, At_mul, U, V, s):
    """One correction sweep from b Ritz triplets (U m x b, V n x b, s):

    R_v = A V - U S and R_u = A^T U - V S (S = diag(s)); the corrections
    F = A^T R_v + R_u S (= A^T A V - V S^2) and E = A F + R_v S^2
    (= A A^T A V - U S^3), each scaled to unit column inf-norm (Sec. 2) and
    projected against the Ritz vectors (F - V (V^T F), E - U (U^T E));
    Algorithm 8 on both; Algorithm 5 over S_u = [U, E], S_v = [V, F]; the
    sqrt(2) lift of the theorem in Sec. 3.2 for the leading b triplets.
    Returns (s, U, V) of the new triplets, descending."""
    U = np.asarray(U, np.float64)
    V = np.asarray(V, np.float64)
    s = np.asarray(s, np.float64)
    b = U.shape[1]
    Rv = A_mul(V) - U * s
    Ru = At_mul(U) - V * s
    F = At_mul(Rv) + Ru * s
    E = A_mul(F) + Rv * s ** 2
    F = colscale_inf(F)
    E = colscale_inf(E)
    F = F - V @ (V.T @ F)
    E = E - U @ (U.T @ E)
    E = hessenberg(E)[3]
    F = hessenberg(F)[3]
    Su = np.hstack([U, E])
    Sv = np.hstack([V, F])
    sn, Y, Z = pencil_svd(Su.T @ A_mul(Sv), Su.T @ Su, Sv.T @ Sv)
    return sn[:b], math.sqrt(2.0) * (Su @ Y[:, :b]), math.sqrt(2.0) * (Sv @ Z[:, :b])
