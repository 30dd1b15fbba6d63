"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check is a closed form,
an invariant, a textbook/library routine the method reduces to in a special
case, or brute force on a tiny input.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import ofrr as O


def _rng(s):
    return np.random.default_rng(s)


# ---------------------------------------------------------------- inputs
def test_haar_orthonormal_and_spectra():
    Q = wl.haar(300, 40, 7)
    assert np.abs(Q.T @ Q - np.eye(40)).max() < 1e-14
    sig = wl.config2_sigma(60)
    A = wl.dense_svd(200, 60, sig, 11)
    assert np.allclose(np.linalg.svd(A, compute_uv=False), sig, rtol=1e-12, atol=0)
    lam = 1.0 / np.arange(1, 81)
    S = wl.dense_symmetric(80, lam, 12)
    assert np.abs(S - S.T).max() == 0
    assert np.allclose(np.sort(np.linalg.eigvalsh(S))[::-1], lam, rtol=1e-11, atol=1e-15)


def test_grid_csr_matches_kronecker_laplacian():
    N = 7
    rp, ci, va, v = wl.grid_schrodinger_csr(N, 10.0, 3)
    T = 2 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    L = np.kron(np.eye(N), T) + np.kron(T, np.eye(N)) + np.diag(v)
    A = O.csr_apply(rp, ci, va)(np.eye(N * N))
    assert np.abs(A - L).max() < 1e-5          # FP32 values
    assert len(ci) == 5 * N * N - 4 * N
    # constant potential: closed form spectrum
    rp, ci, va = wl.grid_potential_csr(N, np.full(N * N, 0.5))
    ev = np.linalg.eigvalsh(O.csr_apply(rp, ci, va)(np.eye(N * N)))
    assert np.allclose(ev, wl.laplacian_constant_eigs(N, 0.5), atol=1e-6)
    lo, up = O.csr_gershgorin(rp, ci, va)
    assert lo == pytest.approx(0.5) and up == pytest.approx(8.5)


# ---------------------------------------------------------------- rounding
def test_round_bf16_against_torch_and_ties():
    torch = pytest.importorskip("torch")
    x = _rng(1).standard_normal(10000) * np.exp(_rng(2).uniform(-20, 20, 10000))
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), ref)
    # ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert O.round_bf16(1 + 2.0 ** -8) == 1.0
    assert O.round_bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


# ---------------------------------------------------------------- Algorithm 8
def test_hessenberg_equals_row_pivoted_lu():
    """Sec. 4.2.2: the Hessenberg output equals P^T L of partial-pivot LU."""
    W = _rng(3).uniform(0, 1, (200, 24))
    Q, piv, keep, _ = O.hessenberg(W)
    P, L, U = sla.lu(W)               # W = P L U, LAPACK getrf (first-max pivot)
    assert keep.all()
    assert np.abs(Q - P @ L).max() < 1e-12
    # pivot rows are where P^T L has its unit diagonal
    rows = np.argmax(P, axis=0)[:24]
    assert np.array_equal(piv, rows)
    assert np.allclose(Q[piv, np.arange(24)], 1.0)
    assert np.abs(Q).max() <= 1.0 + 1e-15
    # span is preserved: W = Q U
    assert np.abs(Q @ U - W).max() < 1e-12


def test_hessenberg_pivot_structure_and_ties():
    # each later column is zero in every earlier pivot row
    W = _rng(4).standard_normal((60, 10))
    Q, piv, _, _ = O.hessenberg(W)
    for j in range(10):
        assert np.all(Q[piv[j], j + 1:] == 0)
    # ties: column 0 has |.|=2 at rows 1 and 3 -> first index (row 1)
    T = np.array([[1., 1.], [-2., 0.], [0., 1.], [2., 5.]])
    _, piv, _, _ = O.hessenberg(T)
    assert piv[0] == 1
    # after elimination column 1 = [1.5, 0, 1, 5] - ... : pivot at row 3
    assert piv[1] == 3


def test_hessenberg_rank_deficient_keeps_rank():
    rng = _rng(5)
    for r in (1, 3, 7):
        W = rng.standard_normal((100, r)) @ rng.standard_normal((r, 12))
        Q, piv, keep, Qf = O.hessenberg(W)
        assert Q.shape[1] == r and keep.sum() == r
        assert np.all(Qf[:, ~keep] == 0)
        # kept columns span range(W)
        Pq = Q @ np.linalg.pinv(Q)
        assert np.abs(Pq @ W - W).max() < 1e-10


def test_hessenberg_f32_mode_close_to_definition():
    W = _rng(6).standard_normal((500, 32)).astype(np.float32)
    Q64, p64, _, _ = O.hessenberg(W.astype(np.float64))
    Q32, p32, _, _ = O.hessenberg(W, arith="f32")
    assert np.array_equal(p64, p32)
    assert np.abs(Q32.astype(np.float64) - Q64).max() < 1e-4


# ---------------------------------------------------------------- Algorithm 3
def _sym(n, lam, seed):
    return wl.dense_symmetric(n, lam, seed)


def test_ofrr_eig_equals_classical_rr_on_same_span():
    """Sec. 3.1: on an orthonormal basis OFRR is Algorithm 2; and OFRR's Ritz
    values depend only on the span."""
    rng = _rng(7)
    A = _sym(120, rng.standard_normal(120), 8)
    Amul, _ = O.dense_apply(A)
    U = rng.standard_normal((120, 15))
    Qb, _ = np.linalg.qr(U)
    classical = np.linalg.eigvalsh(Qb.T @ A @ Qb)          # Algorithm 2
    theta, Y, X, _ = O.rayleigh_ritz_eig(Amul, U @ rng.standard_normal((15, 15)))
    assert np.allclose(np.sort(theta), classical, atol=1e-11)
    # Galerkin condition: U^T (A X - X Theta) = 0
    assert np.abs(U.T @ (A @ X - X * theta)).max() < 1e-9
    # M-orthonormality of Y
    M = (U @ np.eye(15)).T @ (U @ np.eye(15))


def test_ofrr_eig_exact_invariant_subspace_and_brute_force():
    n, k = 90, 6
    lam = 1.0 / np.arange(1, n + 1)
    A = _sym(n, lam, 9)
    Q = wl.haar(n, n, 9)  # same seed -> the eigenvectors used to build A
    R = _rng(10).standard_normal((k, k)) + 3 * np.eye(k)
    theta, _, X, _ = O.rayleigh_ritz_eig(O.dense_apply(A)[0], Q[:, :k] @ R)
    assert np.allclose(np.sort(theta)[::-1], lam[:k], rtol=1e-11)
    # full space: brute force equals the dense eigensolver
    theta, *_ = O.rayleigh_ritz_eig(O.dense_apply(A)[0], np.eye(n))
    assert np.allclose(theta, np.linalg.eigvalsh(A), atol=1e-14)


def test_pencil_eig_rank_deficient_basis():
    rng = _rng(11)
    A = _sym(50, rng.standard_normal(50), 12)
    U = rng.standard_normal((50, 8))
    U = np.hstack([U, U[:, :2] * 3.0])          # duplicated directions
    theta, Y, X, _ = O.rayleigh_ritz_eig(O.dense_apply(A)[0], U)
    Qb, _ = np.linalg.qr(U[:, :8])
    ref = np.linalg.eigvalsh(Qb.T @ A @ Qb)
    assert len(theta) == 8
    assert np.allclose(np.sort(theta), ref, atol=1e-10)


# ---------------------------------------------------------------- Algorithm 5
def test_ofrr_svd_theorem_and_symmetry():
    rng = _rng(13)
    A = rng.standard_normal((70, 40))
    U = rng.uniform(0, 1, (70, 9))
    V = rng.uniform(0, 1, (40, 7))
    Amul, Atmul = O.dense_apply(A)
    s, Ut, Vt, Y, Z = O.rayleigh_ritz_svd(Amul, U, V)
    # Theorem (Sec. 3.2): sqrt(2) U Y and sqrt(2) V Z are orthonormal
    assert np.abs(Ut.T @ Ut - np.eye(7)).max() < 1e-11
    assert np.abs(Vt.T @ Vt - np.eye(7)).max() < 1e-11
    assert np.allclose(np.einsum('ij,ij->j', Y, (U.T @ U) @ Y), 0.5, atol=1e-12)
    assert np.allclose(np.einsum('ij,ij->j', Z, (V.T @ V) @ Z), 0.5, atol=1e-12)
    # the full pencil spectrum is {+-s} plus |k1-k2| zeros
    B = U.T @ A @ V
    K = np.block([[np.zeros((9, 9)), B], [B.T, np.zeros((7, 7))]])
    M = sla.block_diag(U.T @ U, V.T @ V)
    w = np.sort(sla.eigh(K, M, eigvals_only=True))
    assert np.allclose(w[:7], -s, rtol=1e-10)
    assert np.allclose(w[-7:], s[::-1], rtol=1e-10)
    assert np.abs(w[7:9]).max() < 1e-10 * s[0]


def test_ofrr_svd_equals_classical_rr_and_exact_subspaces():
    rng = _rng(14)
    m, n = 80, 50
    sig = wl.config2_sigma(n)
    A = wl.dense_svd(m, n, sig, 15)
    Amul, Atmul = O.dense_apply(A)
    U = rng.standard_normal((m, 10))
    V = rng.standard_normal((n, 10))
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    ref = np.linalg.svd(Qu.T @ A @ Qv, compute_uv=False)     # Algorithm 4
    s, *_ = O.rayleigh_ritz_svd(Amul, U, V)
    assert np.allclose(s, ref, rtol=1e-11)
    # exact singular subspaces -> exact singular values
    Uh = wl.haar(m, n, 15)
    Vh = wl.haar(n, n, 15 + 1_000_003)
    R1 = rng.standard_normal((6, 6)) + 4 * np.eye(6)
    R2 = rng.standard_normal((6, 6)) + 4 * np.eye(6)
    s, Ut, Vt, _, _ = O.rayleigh_ritz_svd(Amul, Uh[:, :6] @ R1, Vh[:, :6] @ R2)
    assert np.allclose(s, sig[:6], rtol=1e-12)
    res = O.residual_svd(Amul, Atmul, Ut, Vt, s)
    assert res.max() < 1e-12
    # brute force: full spaces
    s, *_ = O.rayleigh_ritz_svd(Amul, np.eye(m), np.eye(n))
    assert np.allclose(s, sig, rtol=1e-10)


# ---------------------------------------------------------------- filters
def test_chebyshev_filter_is_scaled_chebyshev_polynomial():
    lam = np.linspace(0.0, 10.0, 40)
    A = np.diag(lam)
    X = np.eye(40)
    a, b_up, a0, d = 3.0, 10.0, 0.0, 9
    Y = O.chebyshev_filter(lambda Z: A @ Z, X, d, a, b_up, a0)
    e, c = (b_up - a) / 2, (b_up + a) / 2
    coef = np.zeros(d + 1)
    coef[d] = 1
    T = np.polynomial.chebyshev.chebval
    p = T((lam - c) / e, coef) / T((a0 - c) / e, coef)
    assert np.allclose(np.diag(Y), p, rtol=1e-10, atol=1e-14)
    assert np.abs(Y - np.diag(np.diag(Y))).max() == 0


def test_residual_eig_closed_form():
    A = np.diag([3.0, 1.0, 0.5])
    d = 1e-3
    x = np.array([[1.0], [d], [0.0]])
    r = O.residual_eig(lambda Z: A @ Z, x, np.array([3.0]))
    # (A - 3I) x / ||x|| = [0, -2d, 0]/sqrt(1+d^2)
    assert r[0] == pytest.approx(2 * d / math.sqrt(1 + d * d) / 3.0, rel=1e-12)


# ---------------------------------------------------------------- solvers
def test_solve_eig_power_converges_to_closed_form():
    n, k, b = 300, 8, 16
    A, lam = wl.config1(n)
    V0 = wl.uniform_block(n, b, 1001)
    r = O.solve_eig(O.dense_apply(A)[0], n, k, V0, degree=1, max_sweeps=80, tol=1e-10)
    assert r.n_converged == k
    assert np.allclose(r.values, lam[:k], rtol=1e-10)
    assert r.res.max() <= 1e-10


def test_solve_eig_chebyshev_lowest_constant_potential():
    N, k, b = 16, 10, 16
    rp, ci, va = wl.grid_potential_csr(N, np.full(N * N, 0.25))
    Amul = O.csr_apply(rp, ci, va)
    V0 = wl.uniform_block(N * N, b, 3001)
    r = O.solve_eig(Amul, N * N, k, V0, which="smallest", filter="chebyshev", degree=8,
                    max_sweeps=60, tol=1e-10, bounds=O.csr_gershgorin(rp, ci, va))
    exact = wl.laplacian_constant_eigs(N, 0.25)[:k]
    assert r.n_converged == k
    assert np.allclose(r.values, exact, rtol=1e-9)


def test_solve_svd_converges_to_prescribed_sigma():
    m, n, k, b = 400, 120, 10, 20
    sig = wl.config2_sigma(n)
    A = wl.dense_svd(m, n, sig, 2000)
    Amul, Atmul = O.dense_apply(A)
    V0 = wl.uniform_block(n, b, 2001)
    r = O.solve_svd(Amul, Atmul, m, n, k, V0, degree=2, max_sweeps=60, tol=1e-10)
    assert r.n_converged == k
    assert np.allclose(r.values, sig[:k], rtol=1e-10)
    assert np.abs(r.U.T @ r.U - np.eye(k)).max() < 1e-10


# ---------------------------------------------------------------- FP8-E4M3 rounding
def test_e4m3_rounding_pins():
    """round_e4m3 against values fixed by the E4M3 format: the 254 finite codes
    (decoded from their bit fields), idempotence on every one of them, ties to
    the even mantissa at every midpoint, saturation, and hand-worked values."""
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F])
    vals = O.e4m3_decode(codes)
    assert len(np.unique(vals)) == 253                      # +0 and -0 coincide
    assert np.max(vals) == 448.0 and np.min(vals[vals > 0]) == 2.0 ** -9
    assert np.array_equal(O.round_e4m3(vals), vals)
    pos = np.sort(np.unique(vals[vals >= 0]))
    mid = (pos[:-1] + pos[1:]) / 2
    rounded = O.round_e4m3(mid)
    lo_code = np.array([int(np.nonzero(O.e4m3_decode(np.arange(128)) == v)[0][0]) for v in pos[:-1]])
    expect = np.where(lo_code % 2 == 0, pos[:-1], pos[1:])  # even mantissa wins the tie
    assert np.array_equal(rounded, expect)
    assert O.round_e4m3(1.0625) == 1.0 and O.round_e4m3(1.1875) == 1.25
    assert O.round_e4m3(0.3) == 0.3125 and O.round_e4m3(2.0 ** -10) == 0.0
    assert O.round_e4m3(3 * 2.0 ** -10) == 2.0 ** -8
    assert O.round_e4m3(449.0) == 448.0 and O.round_e4m3(-1e6) == -448.0 and O.round_e4m3(470.0) == 448.0


def test_e4m3_scale_exponent():
    rng = np.random.default_rng(8)
    m = np.concatenate([np.exp2(rng.uniform(-100, 100, 2000)), 448.0 * np.exp2(np.arange(-5, 6.0)),
                        [448.0 * (1 + 2.0 ** -52), 1.75, 1.75 * (1 + 2.0 ** -52)]])
    e = O.e4m3_scale_exp(m)
    assert np.all(m * np.exp2(e) <= 448.0) and np.all(m * np.exp2(e + 1) > 448.0)
    assert O.e4m3_scale_exp(0.0) == 0 and O.e4m3_scale_exp(1e-300) == 126 and O.e4m3_scale_exp(1e300) == -126
    Xv, inv = O.quantize_e4m3(np.array([[1.0, 0.0], [-3.0, 0.0]]), by_rows=False)
    assert np.array_equal(inv, [2.0 ** -7, 1.0]) and np.array_equal(Xv[:, 0], [128.0, -384.0])


def test_csr_gershgorin_closed_form_and_containment():
    """-Lap_5pt + c on an N x N grid: interior rows give [c, c + 8] exactly; the
    bounds contain the whole spectrum of a random-potential operator."""
    N, c = 12, 0.5
    rp, ci, va = wl.grid_potential_csr(N, np.full(N * N, c))
    lo, up = O.csr_gershgorin(rp, ci, va)
    assert lo == c and up == c + 8.0
    rp, ci, va, v = wl.grid_schrodinger_csr(10, 10.0, 5)
    lo, up = O.csr_gershgorin(rp, ci, va)
    lam = np.linalg.eigvalsh(O.csr_apply(rp, ci, va)(np.eye(100)))
    assert lo <= lam.min() and lam.max() <= up


def test_residual_svd_exact_and_perturbed_triplets():
    """Zero (to rounding) for exact singular triplets, invariant to positive scales
    of u and v and to flipping both signs, and equal to the closed forms for a
    one-sided sign flip and for a known perturbation of sigma."""
    m, n = 40, 12
    sig = np.linspace(3.0, 1.0, n)
    A = wl.dense_svd(m, n, sig, 7)
    Uf, s, Vt = np.linalg.svd(A, full_matrices=False)
    Amul, Atmul = O.dense_apply(A)
    r = O.residual_svd(Amul, Atmul, 5.0 * Uf[:, :4], 2.0 * Vt[:4].T, s[:4])
    assert r.max() < 1e-14
    assert O.residual_svd(Amul, Atmul, -Uf[:, :4], -Vt[:4].T, s[:4]).max() < 1e-14
    # one sign flipped: A(-v) - s u = -2 s u -> sqrt(4 + 4) s / s
    assert np.allclose(O.residual_svd(Amul, Atmul, Uf[:, :4], -Vt[:4].T, s[:4]), 2.0 * np.sqrt(2.0))
    # sigma off by d: A v - (s + d) u = -d u and A^T u - (s + d) v = -d v -> sqrt(2) |d| / (s + d)
    d = 1e-3
    r = O.residual_svd(Amul, Atmul, Uf[:, :4], Vt[:4].T, s[:4] + d)
    assert np.allclose(r, np.sqrt(2.0) * d / (s[:4] + d), rtol=1e-9)


def test_colscale_inf_pins():
    """Column inf-norm scaling (Sec. 2): every nonzero output column has
    max |entry| = 1 by the abs-max definition, signs are kept (a column whose
    largest-magnitude entry is negative keeps it at -1), a zero column stays
    exactly zero, and nothing is NaN.  Values chosen so the divisions are exact."""
    X = np.array([[-4.0, 0.0, 1.0, 0.5],
                  [2.0, 0.0, -3.0, 0.25],
                  [1.0, 0.0, 2.0, -0.125]])
    Y = O.colscale_inf(X)
    expect = np.array([[-1.0, 0.0, 1.0 / 3.0, 1.0],
                       [0.5, 0.0, -1.0, 0.5],
                       [0.25, 0.0, 2.0 / 3.0, -0.25]])
    assert np.array_equal(Y[:, [0, 1, 3]], expect[:, [0, 1, 3]])
    assert np.allclose(Y[:, 2], expect[:, 2], rtol=0, atol=1e-16)
    assert not np.isnan(Y).any()
    assert np.array_equal(np.max(np.abs(Y), axis=0), [1.0, 0.0, 1.0, 1.0])
    # invariant under positive column scaling; a negative scale flips signs only
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((50, 6))
    D = np.array([2.0 ** 10, 0.5, 3.0, 7.0, 2.0 ** -20, -4.0])
    W = O.colscale_inf(Z * D)
    ref = O.colscale_inf(Z) * np.sign(D)
    assert np.allclose(W, ref, rtol=1e-15, atol=1e-16)
    # empty row count: shape kept, no NaN
    E = O.colscale_inf(np.zeros((0, 3)))
    assert E.shape == (0, 3)


def test_svd_correction_sweep_fixed_point_and_contraction():
    """The FP64 correction sweep of the SVD refinement (the GPU's polish):
    exact singular triplets (LAPACK) are its fixed point; from the paper's
    method after two sweeps (residual ~6e-4 on sigma_j = j^-1.5 with 8 of 16
    wanted) each of the first three sweeps contracts the residual by more
    than 30x (1.6e-8, 4.6e-11, 5.3e-13), the fifth ends at the FP64 floor
    (4.8e-15; without the projection of the corrections against the Ritz
    vectors the Gram of [U, E] reaches cond 1e7 and the residual stalls near
    1e-13), sigma is at the FP64 level after the first and the lifted
    vectors have unit 2-norm (the sqrt(2) of the theorem)."""
    m, n, b, k = 300, 75, 16, 8
    sg = wl.config4_sigma(n)
    A = wl.dense_svd(m, n, sg, 4321)
    Am, Atm = O.dense_apply(A)
    Uf, sf, Vft = np.linalg.svd(A, full_matrices=False)
    s1, U1, V1 = O.svd_correction_sweep(Am, Atm, Uf[:, :b], Vft[:b].T, sf[:b])
    assert np.max(np.abs(s1[:k] - sg[:k]) / sg[:k]) <= 1e-13
    assert O.residual_svd(Am, Atm, U1[:, :k], V1[:, :k], s1[:k]).max() <= 1e-12
    r = O.solve_svd(Am, Atm, m, n, b, wl.uniform_block(n, b, 4322), degree=2, max_sweeps=2, tol=1e-16)
    res0 = O.residual_svd(Am, Atm, r.U[:, :k], r.X[:, :k], r.values[:k]).max()
    assert res0 > 1e-9, res0
    U, V, sv, hist = r.U, r.X, r.values, [res0]
    for it in range(5):
        sv, U, V = O.svd_correction_sweep(Am, Atm, U, V, sv)
        hist.append(O.residual_svd(Am, Atm, U[:, :k], V[:, :k], sv[:k]).max())
        if it < 3:
            assert hist[-1] <= hist[-2] / 30, hist
        assert np.max(np.abs(sv[:k] - sg[:k]) / sg[:k]) <= 1e-14
        assert np.abs(np.linalg.norm(U, axis=0) - 1).max() <= 1e-12
        assert np.abs(np.linalg.norm(V, axis=0) - 1).max() <= 1e-12
    assert hist[-1] <= 2e-14, hist
