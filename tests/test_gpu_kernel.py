"""f3: the matrix-free Gaussian kernel operator (the paper's kernel-matrix
family, Sec. 2 and the kernel-matrix experiments of Sec. 5) on the GPU:
products against the explicit matrix, and the eigen and SVD solvers on it
against LAPACK on the explicit matrix, at the paper's settings (1000 points,
f = 0.2, l = 10, s = 0.01; SVD 1000 x 200 with the second point set a random
subset of the first)."""
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


def dev(a, dtype=None):
    import paper_2505_00281_gb300 as pkg
    t = torch.from_numpy(np.asfortranarray(a)).cuda()
    return pkg.fortran(t.to(dtype) if dtype is not None else t)


@pytest.mark.parametrize("n,b,d", [(1000, 20, 2), (777, 70, 3), (130, 5, 1)])
def test_kernel_apply_against_explicit_matrix(rr, n, b, d):
    f, l, s = 0.2, 10.0, 0.01
    x = wl.kernel_points(n, 6000 + n, d)
    A = wl.gaussian_kernel(n, f, l, s, 6000 + n, d)
    X = np.random.default_rng(n).standard_normal((n, b))
    op = rr.api.kernel_operator(dev(x), f, l, s)
    Y64 = rr.api.rr_kernel_apply(op, dev(X), out_dtype=torch.float64).cpu().numpy()
    ref = A @ X
    absr = np.abs(A) @ np.abs(X)
    assert np.all(np.abs(Y64 - ref) <= 1e-13 * absr + 1e-300)
    Y32 = rr.api.rr_kernel_apply(op, dev(X, torch.float32)).cpu().numpy()
    Xf = X.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(Y32 - A @ Xf) <= (4 * n + 64) * 2.0 ** -24 * (np.abs(A) @ np.abs(Xf)))
    # symmetric operator: A^T X = A X
    Yt = rr.api.rr_kernel_apply(op, dev(X), trans=True, out_dtype=torch.float64).cpu().numpy()
    assert np.all(np.abs(Yt - ref) <= 1e-13 * absr)


def test_kernel_apply_rectangular_both_ways(rr):
    n, m, f, l = 1000, 200, 0.2, 10.0
    x = wl.kernel_points(n, 6100)
    y = x[wl.kernel_subset(n, m, 6101)]
    A = wl.gaussian_kernel_rect(x, y, f, l)
    op = rr.api.kernel_operator(dev(x), f, l, 0.0, Y=dev(y))
    V = np.random.default_rng(1).standard_normal((m, 9))
    U = np.random.default_rng(2).standard_normal((n, 9))
    AV = rr.api.rr_kernel_apply(op, dev(V), out_dtype=torch.float64).cpu().numpy()
    AtU = rr.api.rr_kernel_apply(op, dev(U), trans=True, out_dtype=torch.float64).cpu().numpy()
    assert np.all(np.abs(AV - A @ V) <= 1e-13 * (np.abs(A) @ np.abs(V)))
    assert np.all(np.abs(AtU - A.T @ U) <= 1e-13 * (np.abs(A.T) @ np.abs(U)))


def test_kernel_eig_paper_setting(rr):
    """The 20 largest eigenpairs of the 1000-point kernel matrix (f = 0.2,
    l = 10, s = 0.01), block 32, 3 products per sweep, BF16 basis refined to
    1e-10, through the matrix-free operator."""
    n, f, l, s, k, b = 1000, 0.2, 10.0, 0.01, 20, 32
    x = wl.kernel_points(n, 6200)
    A = wl.gaussian_kernel(n, f, l, s, 6200)
    lam = np.linalg.eigvalsh(A)[::-1][:k]
    op = rr.api.kernel_operator(dev(x), f, l, s)
    p = rr.api.make_params(k, b, 3, 40, 1e-10, basis="bf16", v0=dev(wl.uniform_block(n, b, 6201)), refine=True,
                           phase1_sweeps=2)
    th, X, info = rr.rr_eig(op, p, n)
    th, X = th.cpu().numpy(), X.cpu().numpy()
    assert info["n_converged"] == k, info
    assert np.max(np.abs(th - lam) / lam) <= 1e-10
    assert O.residual_eig(lambda Z: A @ Z, X, th).max() <= 1.5e-10


def test_kernel_svd_paper_setting(rr):
    """The 10 largest singular triplets of the 1000 x 200 kernel matrix (the
    200 points a random subset of the 1000, f = 0.2, l = 10), block 20."""
    n, m, f, l, k, b = 1000, 200, 0.2, 10.0, 10, 24
    x = wl.kernel_points(n, 6300)
    y = x[wl.kernel_subset(n, m, 6301)]
    A = wl.gaussian_kernel_rect(x, y, f, l)
    sig = np.linalg.svd(A, compute_uv=False)[:k]
    op = rr.api.kernel_operator(dev(x), f, l, 0.0, Y=dev(y))
    p = rr.api.make_params(k, b, 2, 40, 1e-10, basis="bf16", v0=dev(wl.uniform_block(m, b, 6302)), refine=True,
                           phase1_sweeps=1)
    s_, U, V, info = rr.rr_svd(op, p)
    s_, U, V = s_.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy()
    assert info["n_converged"] == k, info
    assert np.max(np.abs(s_ - sig) / sig) <= 1e-10
    assert O.residual_svd(lambda Z: A @ Z, lambda Z: A.T @ Z, U, V, s_).max() <= 1.5e-10
