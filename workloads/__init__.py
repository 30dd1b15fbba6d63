"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It
builds operators and start blocks only; it holds none of the method's
arithmetic (no filter, no basis construction, no projection, no solve).

Every generator is deterministic in its seed.  Dense matrices are returned in
column-major (Fortran) order, the layout the paper's GPU code uses (Sec. 5.1).

Workloads (sizes are the full-size cases; tests use smaller instances):

* ``dense_symmetric``  A = Q diag(lam) Q^T with Q Haar-orthogonal (QR of a
  seeded N(0,1) matrix, columns sign-fixed by diag(R) as in Mezzadri 2007).
* ``dense_svd``        A = U diag(sigma) V^T, U and V Haar.
* ``grid_schrodinger_csr``  H = -Laplacian(5-point, Dirichlet) + diag(v) on an
  N x N grid, v_j ~ U[0, vmax] from the seed, CSR with FP32 values.
* ``uniform_block``    the random start block: entries U(0,1) drawn in FP64
  (Sec. 5.2: random initial blocks are drawn from U(0,1) in FP64 and then
  cast to the working precision).
"""
from __future__ import annotations

import math

import numpy as np

# Seeds: configuration c, instance i -> 1000*c + i.
def seed_for(config: int, instance: int = 0) -> int:
    return 1000 * config + instance


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def gaussian(rows: int, cols: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) matrix, FP64, column-major."""
    return np.asfortranarray(_rng(seed).standard_normal((rows, cols)))


def haar(rows: int, cols: int, seed: int) -> np.ndarray:
    """Haar-distributed orthonormal columns: QR of a Gaussian, sign-fixed."""
    q, r = np.linalg.qr(gaussian(rows, cols, seed))
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d)


def dense_symmetric(n: int, lam: np.ndarray, seed: int) -> np.ndarray:
    """A = Q diag(lam) Q^T, symmetrised exactly, FP64 column-major."""
    q = haar(n, n, seed)
    a = (q * lam) @ q.T
    a = 0.5 * (a + a.T)
    return np.asfortranarray(a)


def dense_svd(m: int, n: int, sigma: np.ndarray, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T, m >= n, FP64 column-major; U uses seed, V seed+1."""
    assert m >= n and sigma.shape == (n,)
    u = haar(m, n, seed)
    v = haar(n, n, seed + 1_000_003)
    return np.asfortranarray((u * sigma) @ v.T)


def dense_svd_torch(m: int, n: int, sigma, seed: int, device: str = "cuda"):
    """Same construction as ``dense_svd`` drawn with torch on ``device``.

    Used only for full-size benchmark inputs, where a host QR of a
    16384 x 4096 Gaussian would dominate the run time.  The values differ from
    the numpy draw (different generator); the spectrum is the same by
    construction.  Returns a column-major FP64 tensor (stored as the transpose
    of a contiguous row-major n x m tensor).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))

    def _haar(r, c):
        x = torch.randn(r, c, generator=g, device=device, dtype=torch.float64)
        try:
            q, rr = torch.linalg.qr(x)
        except RuntimeError:
            # some environments (e.g. under a profiler) cannot load torch's
            # device linear-algebra library: factor on the host instead
            q, rr = torch.linalg.qr(x.cpu())
            q, rr = q.to(device), rr.to(device)
        d = torch.sign(torch.diagonal(rr))
        d[d == 0] = 1
        return q * d

    u = _haar(m, n)
    v = _haar(n, n)
    s = torch.as_tensor(np.asarray(sigma), dtype=torch.float64, device=device)
    a = (u * s) @ v.T          # m x n row-major
    # column-major storage of A == row-major storage of A^T
    at = a.T.contiguous()      # n x m row-major; element (i, j) of A at j*m + i
    del u, v, a
    return at


def uniform_block(n: int, b: int, seed: int) -> np.ndarray:
    """Start block V0 with U(0,1) entries, FP64 column-major."""
    return np.asfortranarray(_rng(seed).uniform(0.0, 1.0, size=(n, b)))


def grid_schrodinger_csr(N: int, vmax: float, seed: int):
    """CSR of H = -Lap_5pt + diag(v) on an N x N Dirichlet grid.

    Row index p = y*N + x.  Diagonal 4 + v_p, off-diagonals -1 to the four
    neighbours inside the grid.  Column indices sorted within each row.
    Returns (row_ptr int32 [n+1], col_idx int32 [nnz], values float32 [nnz], v float64 [n]).
    """
    n = N * N
    v = _rng(seed).uniform(0.0, vmax, size=n)
    return _grid_csr(N, 4.0 + v) + (v,)


def grid_potential_csr(N: int, potential: np.ndarray):
    """CSR of -Lap_5pt + diag(potential) (potential length N*N, FP64)."""
    return _grid_csr(N, 4.0 + np.asarray(potential, np.float64))


def _grid_csr(N: int, diag: np.ndarray):
    n = N * N
    p = np.arange(n, dtype=np.int64)
    x = p % N
    y = p // N
    # neighbour lists in sorted column order: up (p-N), left (p-1), self, right (p+1), down (p+N)
    cols = np.stack([p - N, p - 1, p, p + 1, p + N], axis=1)
    valid = np.stack([y > 0, x > 0, np.ones(n, bool), x < N - 1, y < N - 1], axis=1)
    vals = np.stack([-np.ones(n), -np.ones(n), diag, -np.ones(n), -np.ones(n)], axis=1)
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols[valid].astype(np.int32)
    values = vals[valid].astype(np.float32)
    return row_ptr.astype(np.int32), col_idx, values


def laplacian_constant_eigs(N: int, c: float) -> np.ndarray:
    """Closed-form spectrum of -Lap_5pt + c*I on an N x N Dirichlet grid, ascending."""
    t = 2.0 - 2.0 * np.cos(np.arange(1, N + 1) * math.pi / (N + 1))
    return np.sort((t[:, None] + t[None, :]).ravel() + c)


# ---- the five workload recipes -------------------------------------------------

def config1(n: int = 2000):
    """Dense symmetric, lam_i = 1/i, FP64."""
    lam = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    return dense_symmetric(n, lam, seed_for(1)), lam


def config2_sigma(n: int = 4096) -> np.ndarray:
    return np.exp(-np.arange(1, n + 1, dtype=np.float64) / 60.0)


def config4_shapes(count: int = 512, seed: int = 4000):
    """m_i = 4*round(64*16**u_i), u_i ~ U(0,1); n_i = m_i/4."""
    u = _rng(seed).uniform(0.0, 1.0, size=count)
    m = 4 * np.round(64.0 * 16.0 ** u).astype(np.int64)
    return [(int(mi), int(mi // 4)) for mi in m]


def config4_sigma(n: int) -> np.ndarray:
    return np.arange(1, n + 1, dtype=np.float64) ** -1.5


def gaussian_potential(N: int, seed: int, count: int = 8) -> np.ndarray:
    """Learned-warm-start family: V_p on an N x N grid (row index p = y*N + x), a sum of
    `count` Gaussians a_g exp(-|x - c_g|^2 / (2 w_g^2)) with centres uniform in the grid,
    widths uniform in [4, 32] cells and amplitudes uniform in [0, 20].  Returns (N, N) FP64."""
    r = _rng(seed)
    cx = r.uniform(0.0, N, size=count)
    cy = r.uniform(0.0, N, size=count)
    w = r.uniform(4.0, 32.0, size=count)
    a = r.uniform(0.0, 20.0, size=count)
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    v = np.zeros((N, N))
    for g in range(count):
        v += a[g] * np.exp(-((x - cx[g]) ** 2 + (y - cy[g]) ** 2) / (2.0 * w[g] ** 2))
    return v


def conv_params(layers, seed: int):
    """He-uniform initial weights and zero biases for a stack of 3x3 convolutions:
    layers = [(cin, cout), ...]; returns [(W (cout, cin, 3, 3) FP32, b (cout,) FP32), ...]."""
    r = _rng(seed)
    out = []
    for cin, cout in layers:
        lim = math.sqrt(6.0 / (cin * 9))
        out.append((r.uniform(-lim, lim, size=(cout, cin, 3, 3)).astype(np.float32),
                    np.zeros(cout, dtype=np.float32)))
    return out


def kernel_points(n: int, seed: int, d: int = 2) -> np.ndarray:
    """n points drawn uniformly from the cube of side sqrt(n) in d dimensions
    (the square for d = 2: one point per unit area at every n), n x d FP64."""
    return np.asfortranarray(_rng(seed).uniform(0.0, math.sqrt(n), size=(n, d)))


def kernel_subset(n: int, m: int, seed: int) -> np.ndarray:
    """m distinct indices of n points, drawn without replacement (the second
    point set of the paper's kernel SVD: a random subset of the first)."""
    return np.sort(_rng(seed).choice(n, size=m, replace=False))


def gaussian_kernel(n: int, f: float, l: float, s: float, seed: int, d: int = 2) -> np.ndarray:
    """Gaussian kernel matrix A_ij = f (exp(-|x_i - x_j|^2 / (2 l^2)) + s delta_ij) over n points
    drawn uniformly from the square (d = 2) of side sqrt(n), the paper's kernel-matrix family
    (1000 points, f = 1 or 0.2, l = 1 ... 100, s = 0.01 or 0).  FP64, column-major."""
    x = kernel_points(n, seed, d)
    d2 = np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=-1)
    return np.asfortranarray(f * (np.exp(-d2 / (2.0 * l * l)) + s * np.eye(n)))


def gaussian_kernel_rect(x: np.ndarray, y: np.ndarray, f: float, l: float) -> np.ndarray:
    """A_ij = f exp(-|x_i - y_j|^2 / (2 l^2)) between two point sets (the
    kernel SVD setting), FP64 column-major."""
    d2 = np.sum((x[:, None, :] - y[None, :, :]) ** 2, axis=-1)
    return np.asfortranarray(f * np.exp(-d2 / (2.0 * l * l)))


def block_diag_csr(n: int, k: int, seed: int):
    """Symmetric CSR made of 4 x 4 diagonal blocks Q diag(e) Q^T (Q random
    orthogonal): the k + 8 largest eigenvalues spread over [0.6, 1], the rest
    in [0, 0.2].  Values are stored in FP32; the exact spectrum is that of the
    stored blocks (brute force per block, FP64)."""
    rng = _rng(seed)
    e = rng.uniform(0.0, 0.2, n)
    e[rng.permutation(n)[:k + 8]] = np.linspace(1.0, 0.6, k + 8)
    nb = n // 4
    Q, _ = np.linalg.qr(rng.standard_normal((nb, 4, 4)))
    B = (Q * e.reshape(nb, 1, 4)) @ np.swapaxes(Q, 1, 2)
    B = 0.5 * (B + np.swapaxes(B, 1, 2))
    B32 = B.astype(np.float32)
    lam = np.sort(np.linalg.eigvalsh(B32.astype(np.float64)).ravel())[::-1]
    rp = np.arange(0, 4 * n + 1, 4, dtype=np.int32)
    ci = (4 * np.repeat(np.arange(nb), 16) + np.tile(np.tile(np.arange(4), 4), nb)).astype(np.int32)
    return rp, ci, B32.reshape(-1), lam
