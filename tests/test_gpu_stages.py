"""Parity of each hot-path stage (CUDA, through the C ABI) with the FP64 oracle.

Integer/byte work (casts to BF16, Hessenberg pivots and FP32 arithmetic) is
compared bit for bit; floating-point accumulations within the error bound of
the arithmetic they use (stated per test).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import ofrr as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rr():
    import paper_2505_00281_gb300 as pkg
    from paper_2505_00281_gb300 import build

    build.build()
    pkg.lib()
    return pkg


DEV = "cuda"
U24 = 2.0 ** -24
U53 = 2.0 ** -53


def dev(a, dtype=None):
    t = torch.from_numpy(np.asfortranarray(a)).to(DEV)
    if dtype is not None:
        t = t.to(dtype)
    import paper_2505_00281_gb300 as pkg
    return pkg.fortran(t)


def host(t):
    return t.detach().to(torch.float64).cpu().numpy()


# ---------------------------------------------------------------- a1
@pytest.mark.parametrize("rows,cols", [(1000, 16), (257, 3), (1, 5)])
def test_colscale_cast_bitexact(rr, rows, cols):
    X = wl.uniform_block(rows, cols, 1001) - 0.3
    X[:, 0] = 0.0  # zero column stays zero
    for dt, rnd in ((torch.bfloat16, O.round_bf16), (torch.float32, lambda a: a.astype(np.float32).astype(np.float64)),
                    (torch.float64, lambda a: a)):
        Y, sc = rr.rr_colscale_cast(dev(X), dt)
        ref = rnd(O.colscale_inf(X))
        assert np.array_equal(host(Y), ref)
        assert np.array_equal(host(sc), np.abs(X).max(axis=0))


def test_cast_operator_bitexact(rr):
    A = wl.gaussian(333, 130, 5)
    col, row = rr.rr_cast_operator(dev(A), torch.bfloat16)
    ref = O.round_bf16(A)
    assert np.array_equal(host(col), ref)
    assert np.array_equal(host(row).reshape(333, 130), ref)   # row-major copy


def _bf16_bits_ref(x):
    return (O.round_bf16(x).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)


def _bf16_bits(t):
    return t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("m,n", [(300, 136), (77, 29)])
def test_split_operator_bitexact(rr, m, n):
    """hi = bf16(A), lo = bf16(A - hi) with the oracle's cast (FP64 -> FP32 -> BF16, nearest even
    both times), bit for bit, column- and row-major: Gaussian entries plus ties at either rounding,
    signed zeros, wide exponents and remainders below FP32's normal range."""
    A = wl.gaussian(m, n, 11 + m)
    t24, t8 = 2.0 ** -24, 2.0 ** -8
    special = [1 + t8, 1 + 3 * t8, 1 + t8 + t24, 1 + t8 + t24 + 2.0 ** -40, -(1 + t8 + t24), 0.0, -0.0,
               2.0 ** 100 * (1 + 2.0 ** -9 + 2.0 ** -30), 2.0 ** -120 * (1 + 2.0 ** -9 + 2.0 ** -30),
               -(2.0 ** -118) * (1 + 2.0 ** -12 + 2.0 ** -33), 1.5 * 2.0 ** -126, 2.0 ** -130, 3.0e38, 1e-300]
    A[: len(special), 0] = special
    A[1, 1: 1 + len(special)] = special[: n - 1]
    hc, hr, lc, lr = rr.rr_split_operator(dev(A))
    hi = O.round_bf16(A)
    hb, lb = _bf16_bits_ref(A), _bf16_bits_ref(A - hi)
    assert np.array_equal(_bf16_bits(hc.t()).reshape(n, m).T, hb)
    assert np.array_equal(_bf16_bits(lc.t()).reshape(n, m).T, lb)
    assert np.array_equal(_bf16_bits(hr).reshape(m, n), hb)
    assert np.array_equal(_bf16_bits(lr).reshape(m, n), lb)


_TDT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


@pytest.mark.parametrize("n,p1,p2,b,t1,t2", [
    (16384, 128, 128, 128, "f64", "f32"),   # the refinement's [X, D] Y at the SVD workload's size
    (4096, 128, 0, 128, "bf16", None),      # phase-1 lift of a BF16 basis
    (1000, 64, 40, 72, "f64", "bf16"),      # ragged rows and columns
    (777, 30, 5, 17, "f32", "f64")])        # K = 35 (not a multiple of 8): FP64-arithmetic path
def test_lift_fp64_accurate(rr, n, p1, p2, b, t1, t2):
    """X = [S1 S2] Y against an FP64 reference: exact on integer data (every slice product and sum
    is exact, so the tensor-core lift must reproduce the exact result), and within K 2^-40 of
    max|row| max|col| on full-mantissa data with row and column scales spread over 2^+-20."""
    rng = np.random.default_rng(n + p1 + b)
    K = p1 + p2
    for integer in (True, False):
        if integer:
            S = rng.integers(-2 ** 20, 2 ** 20, size=(n, K)).astype(np.float64)
            Y = rng.integers(-2 ** 20, 2 ** 20, size=(K, b)).astype(np.float64)
            if t1 == "bf16" or t2 == "bf16":
                S = np.round(S / 2 ** 13)          # 8 significant bits: exact in BF16
        else:
            S = rng.standard_normal((n, K)) * np.exp2(rng.integers(-20, 21, size=(n, 1)))
            Y = rng.standard_normal((K, b)) * np.exp2(rng.integers(-20, 21, size=(1, b)))
        S1d = dev(S[:, :p1], _TDT[t1])
        S2d = dev(S[:, p1:], _TDT[t2]) if t2 else None
        Sh = np.hstack([host(S1d)] + ([host(S2d)] if t2 else []))   # the values as stored
        X = host(rr.rr_lift(S1d, dev(Y), S2d))
        ref = Sh @ Y
        if integer:
            assert np.array_equal(X, ref)
        else:
            bound = K * 2.0 ** -40 * np.abs(Sh).max(axis=1)[:, None] * np.abs(Y).max(axis=0)[None, :]
            assert np.all(np.abs(X - ref) <= bound)


# ---------------------------------------------------------------- a2
@pytest.mark.parametrize("M,N,K", [(300, 40, 700), (128, 128, 4096), (1000, 7, 33),
                                   # tcgen05 path: ragged M, K tail, N padded to 16, K-split
                                   (1000, 128, 2048), (300, 40, 520), (4096, 128, 16384),
                                   (16384, 128, 4096), (2048, 256, 1024)])
def test_gemm_lowp_bf16_within_fp32_bound(rr, M, N, K):
    """C = A_k^T B (+ coef R) within the FP32 recursive-summation bound
    K u32 |A|^T |B| (tensor-core and SIMT paths; lda % 8 == 0 takes tcgen05)."""
    rng = np.random.default_rng(M + N + K)
    Ak = O.round_bf16(rng.standard_normal((K, M)))       # K x M, K-contiguous
    B = O.round_bf16(rng.standard_normal((K, N)))
    R = rng.standard_normal((M, N))
    coef = rng.standard_normal(N)
    C = rr.rr_gemm_lowp(2, M, N, K, dev(Ak, torch.bfloat16), K, dev(B, torch.bfloat16), K,
                        R=dev(R), coef=dev(coef))
    ref = Ak.T @ B + R * coef
    bound = K * U24 * (np.abs(Ak).T @ np.abs(B)) + 2 * U24 * np.abs(R * coef) + 1e-30
    err = np.abs(host(C) - ref)
    assert np.all(err <= 2 * bound), (err / bound).max()


def test_gemm_f64_both_layouts(rr):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((250, 90))
    B = rng.standard_normal((90, 17))
    C = rr.rr_gemm_f64(0, dev(A), dev(B))
    bound = 90 * U53 * (np.abs(A) @ np.abs(B))
    assert np.all(np.abs(host(C) - A @ B) <= 2 * bound)
    B2 = rng.standard_normal((250, 9))
    C2 = rr.rr_gemm_f64(1, dev(A), dev(B2))
    bound = 250 * U53 * (np.abs(A).T @ np.abs(B2))
    assert np.all(np.abs(host(C2) - A.T @ B2) <= 2 * bound)


@pytest.mark.parametrize("trans,M,N,K", [(0, 1000, 64, 512), (1, 512, 128, 16384), (0, 16384, 128, 4096),
                                         (1, 4096, 128, 16384), (0, 256, 40, 1024)])
def test_gemm_f64_emulated_matches_fp64(rr, trans, M, N, K):
    """Error-free BF16 slicing on the tensor cores.  8 slices of 6 bits carry
    every entry to 2^-49 of its row's (op(A)) or column's (B) largest |entry|;
    the slice products are exact, so the error is that representation error
    plus FP64 rounding of the summation:
      |err| <= 2^-48 (rowmax_i sum_j |b_jc| + colmax_c sum_j |a_ij|) + 64 u64 (|A||B|)_ic."""
    rng = np.random.default_rng(M + N + K + trans)
    A = rng.standard_normal((K, M) if trans else (M, K)) * np.exp(rng.uniform(-3, 3, (1, M) if trans else (M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-2, 2, (1, N)))
    C = rr.rr_gemm_f64_emulated(trans, dev(A), dev(B))
    Aop = A.T if trans else A
    ref = Aop @ B
    rowmax = np.abs(Aop).max(axis=1)[:, None]
    colmax = np.abs(B).max(axis=0)[None, :]
    bound = 2.0 ** -48 * (rowmax * np.abs(B).sum(axis=0)[None, :] + colmax * np.abs(Aop).sum(axis=1)[:, None]) \
        + 64 * U53 * (np.abs(Aop) @ np.abs(B))
    err = np.abs(host(C) - ref)
    assert np.all(err <= bound), (err / bound).max()
    # and it is far more accurate than the FP32-accumulated product
    assert np.max(err / (np.abs(Aop) @ np.abs(B))) < 1e-12


@pytest.mark.parametrize("trans", [0, 1])
def test_f64_emulation_exact_on_integers(rr, trans):
    """Integer operands that the slices carry exactly (|entries| < 2^15, so
    every entry is a multiple of its row's or column's 2^-48 slice unit) and
    whose exact products stay below 2^53: the tensor-core sums, the FP32
    accumulation over K chunks, the epilogue's integer combination and the
    FP64 additions are then all exact, so the emulated product must equal the
    integer product bit for bit.  Also pins the Gram path (both operands
    sliced) the same way.  K spans several 4096-long chunks and a ragged
    tail."""
    rng = np.random.default_rng(77 + trans)
    M, N, K = 304, 96, 9000
    A = rng.integers(-2 ** 15 + 1, 2 ** 15, (K, M) if trans else (M, K)).astype(np.int64)
    B = rng.integers(-2 ** 15 + 1, 2 ** 15, (K, N)).astype(np.int64)
    ref = (A.T if trans else A) @ B  # |ref| < 9000 * 2^30 < 2^44: exact in FP64
    C = rr.rr_gemm_f64_emulated(trans, dev(A.astype(np.float64)), dev(B.astype(np.float64)))
    assert np.array_equal(host(C), ref.astype(np.float64))
    X = rng.integers(-2 ** 15 + 1, 2 ** 15, (K, 130)).astype(np.int64)
    G = rr.rr_gram(dev(X.astype(np.float64)), dev(B.astype(np.float64)))
    assert np.array_equal(host(G), (X.T @ B).astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(16384, 128, 4096), (4096, 128, 16384), (1000, 100, 777 + 7)])
def test_gemm_lowp_split_two_term_accuracy(rr, M, N, K):
    """Split-BF16 product (A_hi + A_lo)^T (B_hi + B_lo) without lo.lo, FP32
    accumulation: the error against the exact product of the wide operands is
    the dropped term plus the residual of the 16-bit pairs and FP32 rounding,
    |err| <= (3 u_bf16^2 + 4 K u32) (|A|^T |B|), about 1000x below the plain
    BF16 product's error; the K-split path is taken for small M."""
    rng = np.random.default_rng(M + N + K)
    K = K - K % 8
    A = rng.standard_normal((K, M)).astype(np.float32).astype(np.float64)
    B = rng.standard_normal((K, N)).astype(np.float32).astype(np.float64)
    Ah, Bh = O.round_bf16(A), O.round_bf16(B)
    Al, Bl = O.round_bf16(A - Ah), O.round_bf16(B - Bh)
    dA = lambda X: rr.fortran(torch.from_numpy(np.asfortranarray(X)).to(DEV).to(torch.bfloat16))
    C = rr.rr_gemm_lowp_split(M, N, K, dA(Ah), dA(Al), K, dA(Bh), dA(Bl), K)
    ref = A.T @ B
    absr = np.abs(A).T @ np.abs(B)
    err = np.abs(host(C) - ref)
    assert np.all(err <= (3 * 2.0 ** -16 + 4 * K * U24) * absr + 1e-30)
    plain = np.abs(Ah.T @ Bh - ref)
    assert np.median(err) < 0.05 * np.median(plain)


# ---------------------------------------------------------------- a4 (Algorithm 8)
@pytest.mark.parametrize("n,k", [(1000, 48), (20000, 32), (77, 77), (5, 3),
                                 (16384, 128), (4096, 128), (65536, 160)])
def test_hessenberg_bitexact_fp32(rr, n, k):
    """Pivots and basis bit for bit against the oracle's FP32 process, up to
    the shapes the solvers run: 16384 x 128 (the dense SVD's A V blocks, a
    cooperative grid), 4096 x 128 (its A^T U blocks, one thread-block cluster)
    and 65536 x 160 (a tall block of the sparse workload's width)."""
    W = np.random.default_rng(n + k).standard_normal((n, k)).astype(np.float32)
    Qo, pivo, keepo, Qfo = O.hessenberg(W, arith="f32")
    Wd = dev(W.astype(np.float64), torch.float32)
    Q, piv, err = rr.rr_hessenberg(Wd, qtype=torch.float32)
    assert int(err.cpu()[0]) == 0
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(Q.cpu().numpy(), Qfo)


@pytest.mark.parametrize("n,k,panel", [(16384, 128, 16), (4096, 128, 8), (20000, 100, 32), (3000, 40, 7),
                                       (16, 40, 16)])
def test_hessenberg_blocked_bitexact(rr, n, k, panel):
    """The blocked (level-3) process in panels of r columns against the
    unblocked FP32 oracle, bit for bit (pivots and basis), at the dense SVD's
    block shapes, ragged last panels and a block wider than tall (its later
    columns are all skipped)."""
    W = np.random.default_rng(n + k + panel).standard_normal((n, k)).astype(np.float32)
    Qo, pivo, keepo, Qfo = O.hessenberg(W, arith="f32")
    Q, piv, err = rr.rr_hessenberg_blocked(dev(W.astype(np.float64), torch.float32), panel, qtype=torch.float32)
    assert int(err.cpu()[0]) == 0
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(Q.cpu().numpy(), Qfo)


def test_hessenberg_blocked_ties_rank_deficiency(rr):
    """Integer block with repeated maxima and dependent columns inside and
    across panels: the same pivots, skips and BF16 basis as the oracle."""
    rng = np.random.default_rng(19)
    W = rng.integers(-3, 4, size=(2000, 40)).astype(np.float32)
    W[:, 5] = W[:, 1] + W[:, 2]
    W[:, 21] = W[:, 3] - W[:, 17]
    Qo, pivo, keepo, Qfo = O.hessenberg(W, arith="f32")
    assert not keepo[5] and not keepo[21]
    Q, piv, err = rr.rr_hessenberg_blocked(dev(W.astype(np.float64), torch.float32), 16, qtype=torch.bfloat16)
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(host(Q), O.round_bf16(Qfo))


def test_hessenberg_tall_block_of_the_sparse_workload(rr):
    """1,048,576 x 160 (the sparse workload's basis block: the default entry
    takes the blocked path there), pivots and basis bit for bit against the
    oracle's FP32 process, and the panel form of the oracle (FP64, exact
    arithmetic equal to Algorithm 8) giving the same pivots."""
    from oracle import krylov as OK
    n, k = 1 << 20, 160
    W = np.random.default_rng(1160).standard_normal((n, k)).astype(np.float32)
    Qo, pivo, keepo, Qfo = O.hessenberg(W, arith="f32")
    Q, piv, err = rr.rr_hessenberg(dev(W.astype(np.float64), torch.float32), qtype=torch.float32)
    assert int(err.cpu()[0]) == 0
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(Q.cpu().numpy(), Qfo)
    Qb, pivb = OK.hessenberg_blocked(W[:65536].astype(np.float64), 16)
    Qu, pivu, _, _ = O.hessenberg(W[:65536].astype(np.float64))
    assert np.array_equal(pivb, pivu)


def test_hessenberg_ties_rank_deficiency_and_bf16_output(rr):
    # integer-valued block with repeated maxima and an exactly dependent column
    rng = np.random.default_rng(9)
    W = rng.integers(-3, 4, size=(600, 12)).astype(np.float32)
    W[:, 5] = W[:, 1] + W[:, 2]
    Qo, pivo, keepo, Qfo = O.hessenberg(W, arith="f32")
    assert not keepo[5]
    Q, piv, err = rr.rr_hessenberg(dev(W.astype(np.float64), torch.float32), qtype=torch.bfloat16)
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(host(Q), O.round_bf16(Qfo))


def test_hessenberg_fp64_matches_lu(rr):
    import scipy.linalg as sla
    W = np.random.default_rng(11).uniform(0, 1, (3000, 40))
    Q, piv, err = rr.rr_hessenberg(dev(W), qtype=torch.float64)
    P, L, U = sla.lu(W)
    assert np.abs(host(Q) - P @ L).max() < 1e-12
    Qo, pivo, _, Qfo = O.hessenberg(W)
    assert np.array_equal(piv.cpu().numpy().astype(np.int64), pivo)
    assert np.array_equal(host(Q), Qfo)


# ---------------------------------------------------------------- a5
def test_gram_fp64_accurate_mixed_types(rr):
    rng = np.random.default_rng(12)
    n = 5000
    X = O.round_bf16(rng.standard_normal((n, 37)))
    Y = rng.standard_normal((n, 50))
    G = rr.rr_gram(dev(X, torch.bfloat16), dev(Y))
    ref = X.T @ Y
    bound = n * U53 * (np.abs(X).T @ np.abs(Y))
    assert np.all(np.abs(host(G) - ref) <= 2 * bound)
    G2 = rr.rr_gram(dev(Y), dev(Y))
    assert np.all(np.abs(host(G2) - Y.T @ Y) <= 2 * n * U53 * (np.abs(Y).T @ np.abs(Y)))


@pytest.mark.parametrize("n,p,q", [(8200, 130, 100), (4104, 40, 300)])
def test_gram_tensor_core_path_wide_range(rr, n, p, q):
    """The tensor-core Gram path (n % 8 == 0; Y in column chunks of at most
    128): ragged tiles, a K range that is not a multiple of the 4096-long
    exact chunks, columns spanning many binades and rows far below the column
    maxima, mixed storage types and accumulation.  Bound: the slice truncation
    (2^-47 n times the column maxima) plus the FP64 reference's own rounding."""
    rng = np.random.default_rng(31)
    X = rng.standard_normal((n, p)) * np.exp2(rng.integers(-30, 30, p))[None, :]
    X[rng.random((n, p)) < 0.3] *= 1e-9
    Y = rng.standard_normal((n, q)) * np.exp2(rng.integers(-20, 20, q))[None, :]
    ref = X.T @ Y
    tail = 2 * n * U53 * (np.abs(X).T @ np.abs(Y))
    trunc = 2.0 ** -47 * n * np.outer(np.abs(X).max(0), np.abs(Y).max(0))
    G = host(rr.rr_gram(dev(X), dev(Y)))
    assert np.all(np.abs(G - ref) <= trunc + tail)
    # mixed types: BF16 X, FP32 Y, accumulated onto an existing G
    Xb = O.round_bf16(X)
    Yf = Y.astype(np.float32).astype(np.float64)
    G0 = rng.standard_normal((p, q))
    Gd = dev(G0)
    rr.rr_gram(dev(Xb, torch.bfloat16), dev(Yf, torch.float32), G=Gd, accumulate=True)
    ref2 = G0 + Xb.T @ Yf
    bound2 = 2.0 ** -47 * n * np.outer(np.abs(Xb).max(0), np.abs(Yf).max(0)) + 2 * n * U53 * (
        np.abs(G0) + np.abs(Xb).T @ np.abs(Yf))
    assert np.all(np.abs(host(Gd) - ref2) <= bound2)


# ---------------------------------------------------------------- a6
@pytest.mark.parametrize("b", [16, 64, 129])
def test_pencil_eig_matches_generalized_eigensolver(rr, b):
    import scipy.linalg as sla
    rng = np.random.default_rng(b)
    U = rng.uniform(0, 1, (4 * b, b))
    S = rng.standard_normal((4 * b, 4 * b))
    A = S + S.T
    H = U.T @ A @ U
    G = U.T @ U
    th, Y, dropped = rr.rr_pencil_eig(dev(H), dev(G))
    ref = sla.eigh(H, G, eigvals_only=True)
    th = host(th)
    assert dropped == 0
    scale = np.abs(ref).max()
    assert np.abs(th - ref).max() <= 1e-10 * scale
    Yh = host(Y)
    assert np.abs(Yh.T @ G @ Yh - np.eye(b)).max() < 1e-8
    assert np.abs(H @ Yh - G @ Yh * th).max() < 1e-8 * scale


@pytest.mark.parametrize("b", [144, 160, 320])
def test_pencil_eig_positive_spectrum_dense_whitened(rr, b):
    """A pencil whose whitened matrix C = L^-1 H L^-T is dense with a positive
    spectrum in [0.16, 0.86] (a BF16 power-filtered basis gives such pencils):
    the Gershgorin interval of C reaches far below the spectrum, and the shift
    must still keep the Jacobi's singular values apart.  G has condition
    ~5e5.  Exact values by construction; the oracle's generalized eigensolver
    as the second reference."""
    import scipy.linalg as sla
    rng = np.random.default_rng(7300 + b)
    Q, _ = np.linalg.qr(rng.standard_normal((b, b)))
    theta = np.sort(rng.uniform(0.16, 0.86, b))
    C = (Q * theta) @ Q.T
    Bq, _ = np.linalg.qr(rng.standard_normal((b, b)))
    G = (Bq * np.logspace(0, np.log10(5e5), b)) @ Bq.T
    G = 0.5 * (G + G.T)
    L = np.linalg.cholesky(G)
    H = L @ C @ L.T
    H = 0.5 * (H + H.T)
    th, Y, dropped = rr.rr_pencil_eig(dev(H), dev(G))
    th, Yh = host(th), host(Y)
    ref = sla.eigh(H, G, eigvals_only=True)
    assert dropped == 0
    assert np.abs(th - ref).max() <= 1e-10
    assert np.abs(th - theta).max() <= 1e-9
    assert np.abs(Yh.T @ G @ Yh - np.eye(b)).max() < 1e-8
    assert np.abs(H @ Yh - G @ Yh * th).max() < 1e-8 * np.abs(H).max()


def test_pencil_eig_rank_deficient_drops(rr):
    rng = np.random.default_rng(5)
    U = rng.standard_normal((80, 10))
    U = np.hstack([U, U[:, :3]])
    S = rng.standard_normal((80, 80))
    A = S + S.T
    th, Y, dropped = rr.rr_pencil_eig(dev(U.T @ A @ U), dev(U.T @ U))
    th = host(th)
    assert dropped == 3
    ref, *_ = O.rayleigh_ritz_eig(lambda Z: A @ Z, U)
    assert np.all(np.isnan(th[10:]))
    assert np.allclose(th[:10], ref, atol=1e-9)


@pytest.mark.parametrize("b1,b2", [(32, 32), (64, 48), (130, 130)])
def test_pencil_svd_matches_block_pencil(rr, b1, b2):
    rng = np.random.default_rng(b1 * b2)
    A = rng.standard_normal((300, 200))
    U = rng.uniform(0, 1, (300, b1))
    V = rng.uniform(0, 1, (200, b2))
    B, Gu, Gv = U.T @ A @ V, U.T @ U, V.T @ V
    s, Y, Z, dropped = rr.rr_pencil_svd(dev(B), dev(Gu), dev(Gv))
    so, Yo, Zo = O.pencil_svd(B, Gu, Gv)          # literal 2x2 block pencil (Algorithm 5)
    s = host(s)
    assert np.allclose(s, so, rtol=1e-9, atol=1e-12 * so[0])
    Ut = U @ host(Y)
    Vt = V @ host(Z)
    r = min(b1, b2)
    assert np.abs(Ut.T @ Ut - np.eye(r)).max() < 1e-8
    assert np.abs(Vt.T @ Vt - np.eye(r)).max() < 1e-8


@pytest.mark.parametrize("rows", [(600, 500)])
def test_pencil_svd_2b256_random(rr, rows):
    """The dense SVD's refinement pencil size, 2b = 256 on both sides (the
    8-CTA cluster Jacobi and the QR preconditioner on 8 CTAs), against the
    oracle's literal 2x2 block pencil of Algorithm 5 on a random
    non-orthogonal basis."""
    rng = np.random.default_rng(256)
    m, n = rows
    A = rng.standard_normal((m, n))
    U = rng.uniform(0, 1, (m, 256))
    V = rng.uniform(0, 1, (n, 256))
    B, Gu, Gv = U.T @ A @ V, U.T @ U, V.T @ V
    s, Y, Z, dropped = rr.rr_pencil_svd(dev(B), dev(Gu), dev(Gv))
    so, Yo, Zo = O.pencil_svd(B, Gu, Gv)
    s, Yh, Zh = host(s), host(Y), host(Z)
    assert dropped == 0
    assert np.allclose(s, so, rtol=1e-9, atol=1e-12 * so[0])
    assert np.abs(Yh.T @ Gu @ Yh - np.eye(256)).max() < 1e-8
    assert np.abs(Zh.T @ Gv @ Zh - np.eye(256)).max() < 1e-8
    assert np.abs(Yh.T @ B @ Zh - np.diag(s)).max() < 1e-8 * s[0]


def test_pencil_svd_2b256_refinement_pencil(rr):
    """The pencil the dense SVD's refinement solves (2b = 256): S_u = [U~, E],
    S_v = [V~, F] with U~, V~ orthonormal near-singular vectors of A
    (perturbed by 1e-6) and E, F correction blocks at the noise level, so half
    of the 2b singular values sit at the noise floor.  The leading b values
    against the oracle's literal block pencil to 1e-12 of sigma_1 and the
    pencil's defining identities (Y^T Gu Y = I, Z^T Gv Z = I,
    Y^T B Z = diag(s)) to 1e-11."""
    rng = np.random.default_rng(2256)
    m, n, b = 1024, 512, 128
    sig = wl.config2_sigma(n)
    Uh, Vh = wl.haar(m, n, 1), wl.haar(n, n, 2)
    A = (Uh * sig) @ Vh.T
    Ut, _ = np.linalg.qr(Uh[:, :b] + 1e-6 * rng.standard_normal((m, b)))
    Vt, _ = np.linalg.qr(Vh[:, :b] + 1e-6 * rng.standard_normal((n, b)))
    R_v = A @ Vt - Ut * np.sum(Ut * (A @ Vt), axis=0)
    E = R_v + 1e-3 * np.abs(R_v).max() * rng.standard_normal((m, b))
    F = A.T @ E
    F = F - Vt @ (Vt.T @ F)
    E = E / np.abs(E).max(axis=0)
    F = F / np.abs(F).max(axis=0)
    Su, Sv = np.hstack([Ut, E]), np.hstack([Vt, F])
    B, Gu, Gv = Su.T @ A @ Sv, Su.T @ Su, Sv.T @ Sv
    s, Y, Z, dropped = rr.rr_pencil_svd(dev(B), dev(Gu), dev(Gv))
    so, Yo, Zo = O.pencil_svd(B, Gu, Gv)
    s, Yh, Zh = host(s), host(Y), host(Z)
    kept = 2 * b - dropped
    assert kept >= b
    assert np.abs(s[:b] - so[:b]).max() <= 1e-12 * so[0]
    assert np.abs(s[:b] - sig[:b]).max() <= 1e-9 * sig[0]
    eu = np.abs(Yh[:, :b].T @ Gu @ Yh[:, :b] - np.eye(b)).max()
    ev = np.abs(Zh[:, :b].T @ Gv @ Zh[:, :b] - np.eye(b)).max()
    eb = np.abs(Yh[:, :b].T @ B @ Zh[:, :b] - np.diag(s[:b])).max() / s[0]
    print("refinement pencil 2b = 256: orthonormality", eu, ev, "Galerkin", eb)
    assert max(eu, ev, eb) < 1e-11


def _clustered_spectrum(rng, b):
    """Groups of 8 values 1e-6 apart (relative), one exactly degenerate
    group, and well separated singletons: the degenerate case of the pencil
    (the FP32 stage cannot resolve these pairs; the FP64 refinement must)."""
    g = b // 16
    centres = np.linspace(1.0, 3.0, g)
    vals = [c0 * (1 + 1e-6 * rng.standard_normal(8)) for c0 in centres[:-1]]
    vals.append(np.full(8, 3.5))
    vals.append(np.linspace(4.0, 6.0, b - 8 * g))
    return np.concatenate(vals)


@pytest.mark.parametrize("b", [64, 200])
def test_pencil_eig_clustered_spectrum(rr, b):
    import scipy.linalg as sla
    rng = np.random.default_rng(300 + b)
    lam = _clustered_spectrum(rng, b) * rng.choice([-1.0, 1.0])
    Q, _ = np.linalg.qr(rng.standard_normal((b, b)))
    Bm = rng.standard_normal((3 * b, b))
    G = Bm.T @ Bm / (3 * b)
    Lc = np.linalg.cholesky(G)
    H = Lc @ (Q * lam) @ Q.T @ Lc.T
    H = 0.5 * (H + H.T)
    th, Y, dropped = rr.rr_pencil_eig(dev(H), dev(G))
    th, Yh = host(th), host(Y)
    ref = sla.eigh(H, G, eigvals_only=True)
    scale = np.abs(ref).max()
    assert dropped == 0
    assert np.all(np.isfinite(Yh))
    # the same bounds as the unclustered pencil test (FP32-level failures of
    # the refinement show up as 1e-7)
    assert np.abs(np.sort(th) - ref).max() <= 1e-10 * scale
    assert np.abs(Yh.T @ G @ Yh - np.eye(b)).max() < 1e-11
    assert np.abs(H @ Yh - G @ Yh * th).max() < 1e-10 * scale


def test_pencil_svd_clustered_spectrum(rr):
    rng = np.random.default_rng(17)
    b = 160
    sig = _clustered_spectrum(rng, b)
    P, _ = np.linalg.qr(rng.standard_normal((b, b)))
    R, _ = np.linalg.qr(rng.standard_normal((b, b)))
    Bm = (P * sig) @ R.T
    Gu = np.eye(b)
    Gv = np.eye(b)
    s, Y, Z, dropped = rr.rr_pencil_svd(dev(Bm), dev(Gu), dev(Gv))
    s, Yh, Zh = host(s), host(Y), host(Z)
    assert np.all(np.isfinite(Yh)) and np.all(np.isfinite(Zh))
    assert np.abs(s - np.sort(sig)[::-1]).max() <= 1e-10 * sig.max()
    assert np.abs(Yh.T @ Yh - np.eye(b)).max() < 1e-11
    assert np.abs(Zh.T @ Zh - np.eye(b)).max() < 1e-11
    assert np.abs(Bm @ Zh - Yh * s).max() < 1e-10 * sig.max()


# ---------------------------------------------------------------- a3
@pytest.mark.parametrize("b", [20, 160])
def test_chebyshev_step_rows_long_rows(rr, b):
    """Rows with more CSR entries than a CTA stages in shared memory (dense
    rows among sparse ones): those CTAs read their entries from global
    memory.  BF16 blocks against the oracle's CSR product."""
    rng = np.random.default_rng(7400 + b)
    n = 3000
    rows = []
    for i in range(n):
        if i % 500 == 7:
            cols = np.arange(n)                       # a dense row
        else:
            cols = np.unique(np.concatenate([[i], rng.integers(0, n, 4)]))
        rows.append(cols)
    rp = np.concatenate([[0], np.cumsum([len(c) for c in rows])]).astype(np.int32)
    ci = np.concatenate(rows).astype(np.int32)
    va = rng.uniform(-1, 1, len(ci)).astype(np.float32)
    X = O.round_bf16(rng.standard_normal((n, b)))
    Xp = O.round_bf16(rng.standard_normal((n, b)))
    bp = -(-b // 8) * 8

    def rows_(a):
        t = torch.zeros(n, bp, dtype=torch.float64)
        t[:, :b] = torch.from_numpy(a)
        return t.to(torch.bfloat16).to(DEV)
    d_rp, d_ci, d_va = (torch.from_numpy(a).to(DEV) for a in (rp, ci, va))
    alpha, c, beta = 0.7, 3.0, 0.4
    Yn = rr.rr_chebyshev_step_rows(d_rp, d_ci, d_va, rows_(X), rows_(Xp), b, alpha, c, beta, out_dtype=torch.float32)
    Amul = O.csr_apply(rp, ci, va)
    ref = alpha * (Amul(X) - c * X) - beta * Xp
    absb = alpha * (O.csr_apply(rp, ci, np.abs(va))(np.abs(X)) + c * np.abs(X)) + beta * np.abs(Xp)
    got = host(Yn)[:, :b]
    # FP32 sums of a row's terms: the error bound grows with the row's length
    lens = np.diff(rp).astype(np.float64)[:, None]
    assert np.all(np.abs(got - ref) <= (lens + 8) * U24 * absb + 1e-30)


@pytest.mark.parametrize("ytype,otype,b", [("bf16", "bf16", 20), ("bf16", "f32", 160), ("f32", "f32", 13),
                                           ("f64", "f64", 7)])
def test_chebyshev_step_rows(rr, ytype, otype, b):
    """Row-major fused step against the oracle's CSR product, ragged b (pad
    columns up to the 16-byte vector width stay zero), rows without a stored
    diagonal among them (a shift-only row)."""
    N = 40
    rp, ci, va, v = wl.grid_schrodinger_csr(N, 10.0, 3000)
    n = N * N
    # drop the stored diagonal of every seventh row
    keep = np.ones(len(ci), dtype=bool)
    for i in range(0, n, 7):
        e = rp[i] + int(np.nonzero(ci[rp[i]:rp[i + 1]] == i)[0][0])
        keep[e] = False
    ci, va = ci[keep], va[keep]
    rp = np.concatenate([[0], np.cumsum([keep[rp[i]:rp[i + 1]].sum() for i in range(n)])]).astype(rp.dtype)
    tt = {"bf16": torch.bfloat16, "f32": torch.float32, "f64": torch.float64}
    width = 16 // {"bf16": 2, "f32": 4, "f64": 8}[ytype]
    bp = -(-b // width) * width
    rnd = {"bf16": O.round_bf16, "f32": lambda a: a.astype(np.float32).astype(np.float64),
           "f64": lambda a: a}[ytype]
    X = rnd(np.random.default_rng(11).standard_normal((n, b)))
    Xp = rnd(np.random.default_rng(12).standard_normal((n, b)))

    def rows(a):
        t = torch.zeros(n, bp, dtype=torch.float64)
        t[:, :b] = torch.from_numpy(a)
        return t.to(tt[ytype]).to(DEV)
    d_rp, d_ci, d_va = (torch.from_numpy(a).to(DEV) for a in (rp, ci, va))
    alpha, c, beta = 0.7, 3.0, 0.4
    Yn = rr.rr_chebyshev_step_rows(d_rp, d_ci, d_va, rows(X), rows(Xp), b, alpha, c, beta, out_dtype=tt[otype])
    Amul = O.csr_apply(rp, ci, va)
    ref = alpha * (Amul(X) - c * X) - beta * Xp
    got = host(Yn)
    Aabs = O.csr_apply(rp, ci, np.abs(va))           # |A| |X| bounds the rounding of the sums
    absb = alpha * (Aabs(np.abs(X)) + c * np.abs(X)) + beta * np.abs(Xp)
    if ytype == "f64":
        tol = 16 * U53 * absb
    else:
        tol = 16 * U24 * absb + (2.0 ** -8 * np.abs(ref) if otype == "bf16" else 0)
    assert np.all(np.abs(got[:, :b] - ref) <= tol)
    assert np.all(got[:, b:] == 0)
    # first step (no Y_prev)
    Y1 = rr.rr_chebyshev_step_rows(d_rp, d_ci, d_va, rows(X), None, b, alpha, c, 0.0, out_dtype=tt[otype])
    ref1 = alpha * (Amul(X) - c * X)
    absb1 = alpha * (Aabs(np.abs(X)) + c * np.abs(X))
    if ytype == "f64":
        tol1 = 16 * U53 * absb1
    else:
        tol1 = 16 * U24 * absb1 + (2.0 ** -8 * np.abs(ref1) if otype == "bf16" else 0)
    assert np.all(np.abs(host(Y1)[:, :b] - ref1) <= tol1)


def test_csr_spmm_and_chebyshev_step(rr):
    N, b = 40, 24
    rp, ci, va, v = wl.grid_schrodinger_csr(N, 10.0, 3000)
    n = N * N
    Amul = O.csr_apply(rp, ci, va)
    X = O.round_bf16(np.random.default_rng(1).standard_normal((n, b)))
    Xp = O.round_bf16(np.random.default_rng(2).standard_normal((n, b)))
    R = np.random.default_rng(3).standard_normal((n, b))
    gam = np.random.default_rng(4).standard_normal(b)
    bc = np.random.default_rng(5).uniform(0.5, 2, b)
    d_rp, d_ci, d_va = (torch.from_numpy(a).to(DEV) for a in (rp, ci, va))
    Y = rr.rr_csr_spmm(d_rp, d_ci, d_va, dev(X, torch.bfloat16))
    ref = Amul(X)
    assert np.abs(host(Y) - ref).max() <= 8 * U24 * (np.abs(ref).max() + 20)
    alpha, c, beta = 0.7, 3.0, 0.4
    Yn = rr.rr_chebyshev_step(d_rp, d_ci, d_va, dev(X, torch.bfloat16), dev(Xp, torch.bfloat16), alpha, c,
                              beta, beta_col=dev(bc), R=dev(R), gamma=dev(gam), out_dtype=torch.float32)
    ref = alpha * (Amul(X) - c * X) - beta * bc * Xp + gam * R
    assert np.abs(host(Yn) - ref).max() <= 16 * U24 * (np.abs(ref).max() + 40)
    # FP64 path (used for the FP64-accurate residual)
    Xd = np.random.default_rng(6).standard_normal((n, b))
    Y64 = rr.rr_csr_spmm(d_rp, d_ci, d_va, dev(Xd), out_dtype=torch.float64)
    assert np.abs(host(Y64) - Amul(Xd)).max() < 1e-13 * (np.abs(Xd).max() * 20)


# ---------------------------------------------------------------- FP8-E4M3 operands and product
@pytest.mark.parametrize("by_rows", [False, True])
def test_quantize_e4m3_bitexact(rr, by_rows):
    """E4M3 codes and power-of-two scales bit for bit against the oracle's
    rounding (FP32 then E4M3, ties to even, saturation), columns / rows spanning
    many binades, a zero line, a line whose maximum is exactly 448 2^k."""
    rng = np.random.default_rng(41)
    rows, cols = 1000, 37
    X = rng.standard_normal((rows, cols)) * np.exp2(rng.integers(-40, 40, (rows, cols)) // 8)
    X *= np.exp2(rng.integers(-30, 30, cols))[None, :] if not by_rows else np.exp2(rng.integers(-30, 30, rows))[:, None]
    if by_rows:
        X[5, :] = 0.0
        X[7, 3] = 448.0 * 2.0 ** 5
    else:
        X[:, 5] = 0.0
        X[3, 7] = 448.0 * 2.0 ** 5
    Q, inv = rr.rr_quantize_e4m3(dev(X), by_rows=by_rows)
    ref, rinv = O.quantize_e4m3(X, by_rows)
    assert np.array_equal(host(inv), rinv)
    codes = Q.cpu().numpy()
    got = O.e4m3_decode(codes[:, :(cols if by_rows else rows)])
    assert np.array_equal(got, ref if by_rows else ref.T)


@pytest.mark.parametrize("M,N,K", [(300, 40, 1000), (256, 128, 4096)])
def test_gemm_e4m3(rr, M, N, K):
    """tcgen05 kind::f8f6f4 product of E4M3 operands with row / column scales
    against the exact product of the same E4M3 values (FP64), within FP32
    accumulation: K u32 |Q_A| |Q_B| + the two FP32 scale multiplications.
    Ragged M and N tiles, a K tail, and K splits with atomic accumulation."""
    rng = np.random.default_rng(M + K)
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-8, 8, M))[:, None]
    B = rng.standard_normal((K, N))
    Aq, ia = rr.rr_quantize_e4m3(dev(A), by_rows=True)       # rows of A, K contiguous
    Bq, ib = rr.rr_quantize_e4m3(dev(B), by_rows=False)      # columns of B, K contiguous
    C = host(rr.rr_gemm_e4m3(M, N, K, Aq, ia, Bq, ib))
    qa, ra = O.quantize_e4m3(A, True)
    qb, rb = O.quantize_e4m3(B, False)
    ref = ra[:, None] * (qa @ qb) * rb[None, :]
    bound = ra[:, None] * (np.abs(qa) @ np.abs(qb)) * rb[None, :] * K * U24 + 4 * U24 * np.abs(ref)
    assert np.all(np.abs(C - ref) <= bound)
    # the FP8 product approximates the FP64 one to the E4M3 rounding (2^-4 relative per factor)
    assert np.abs(C - A @ B).max() <= 0.25 * (np.abs(A) @ np.abs(B)).max()
