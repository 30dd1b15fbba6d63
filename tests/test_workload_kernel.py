"""The Gaussian kernel-matrix workload (CPU): closed forms at the length-scale
limits, and the oracle's OFRR with the Hessenberg basis on the paper's
double-precision setting (1000 points, f = 0.2, l = 10, s = 0.01; block 50,
3 products per sweep, 10 sweeps, the 20 largest eigenvalues)."""
import numpy as np

import workloads as wl
from oracle import ofrr as O


def test_kernel_matrix_limits():
    n, f, s = 60, 0.7, 0.01
    A = wl.gaussian_kernel(n, f, 1e9, s, 1)           # every pair at distance << l
    lam = np.linalg.eigvalsh(A)
    assert np.allclose(lam[-1], f * (n + s), rtol=1e-12) and np.allclose(lam[:-1], f * s, atol=1e-10)
    B = wl.gaussian_kernel(n, f, 1e-9, s, 1)          # every pair at distance >> l
    assert np.array_equal(B, f * (1 + s) * np.eye(n))
    C = wl.gaussian_kernel(n, f, 3.0, s, 2)
    assert np.array_equal(C, C.T) and np.all(np.diag(C) == f * (1 + s))
    assert np.linalg.eigvalsh(C).min() > 0                # positive definite (s > 0)


def test_oracle_ofrr_on_paper_kernel_setting():
    A = wl.gaussian_kernel(1000, 0.2, 10.0, 0.01, 3)
    V0 = wl.uniform_block(1000, 50, 4)
    res = O.solve_eig(lambda X: A @ X, 1000, 20, V0, degree=3, max_sweeps=10, tol=1e-14)
    exact = np.linalg.eigvalsh(A)[::-1][:20]
    assert np.max(np.abs(res.values[:20] - exact) / exact) < 1e-10
