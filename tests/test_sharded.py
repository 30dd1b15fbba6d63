"""The row-sharded schedule of the method (paper_2505_00281_gb300.sharded) run
as world-size-2 gloo ranks on CPU, each rank holding half of the rows, with
the oracle's FP64 operations as the local compute: the same Ritz values as the
single-rank oracle solve to 1e-12, and the same vectors.  Covers the dense
SVD (A's rows sharded; all-gather before Algorithm 8, partial B and G_U in
one all-reduce) and the CSR eigenproblem (grid lines sharded, halo exchange
of the neighbouring lines in every filter step)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as wl  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """Local compute for the simulation: the oracle's FP64 definitions."""

    def __init__(self):
        from oracle import ofrr as O
        self.O = O

    @staticmethod
    def _t(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))

    def mm(self, A, X):
        return A @ X

    def mm_t(self, A, X):
        return A.T @ X

    def spmm(self, csr, X):
        import scipy.sparse as sp
        M = sp.csr_matrix((csr.values.numpy().astype(np.float64), csr.col_idx.numpy(), csr.row_ptr.numpy()),
                          shape=(csr.row_ptr.shape[0] - 1, X.shape[0]))
        return self._t(M @ X.numpy())

    def basis(self, W):
        return self._t(self.O.hessenberg(W.numpy(), arith="f64")[0])

    def colscale(self, W):
        return self._t(self.O.colscale_inf(W.numpy()))

    def gram(self, X, Y):
        return X.T @ Y

    def pencil_svd(self, B, Gu, Gv):
        s, Y, Z = self.O.pencil_svd(B.numpy(), Gu.numpy(), Gv.numpy())
        return self._t(s), self._t(np.sqrt(2.0) * Y), self._t(np.sqrt(2.0) * Z)

    def pencil_eig(self, H, G):
        th, Y = self.O.pencil_eig(H.numpy(), G.numpy())
        return self._t(th), self._t(Y)

    def colnorm2(self, R):
        return (R * R).sum(dim=0)


def _svd_worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2505_00281_gb300 import sharded as S

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, n, b, k = 600, 200, 16, 8
    A = wl.dense_svd(m, n, wl.config2_sigma(n), 5100)
    V0 = wl.uniform_block(n, b, 5101)
    rows = S.row_partition(m, world)
    s0, s1 = rows[rank]
    r = S.svd_sharded(OracleOps(), torch.from_numpy(np.ascontiguousarray(A[s0:s1])), m, n, k,
                      torch.from_numpy(np.ascontiguousarray(V0)), degree=2, sweeps=3, rows=rows)
    out[rank] = (r.values.numpy(), r.X.numpy(), r.U.numpy(), r.res.numpy(), (s0, s1))
    dist.barrier()
    dist.destroy_process_group()


def _eig_worker(rank, world, port, out):
    import torch.distributed as dist
    from oracle import ofrr as O
    from paper_2505_00281_gb300 import sharded as S

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    N, b, k = 24, 12, 6
    rp, ci, va, _ = wl.grid_schrodinger_csr(N, 10.0, 5200)
    V0 = wl.uniform_block(N * N, b, 5201)
    lines = S.grid_partition(N, world)
    y0, y1 = lines[rank]
    csr = S.local_csr(torch.from_numpy(rp.astype(np.int64)), torch.from_numpy(ci.astype(np.int64)),
                      torch.from_numpy(va), N, y0, y1)
    r = S.eig_csr_sharded(OracleOps(), csr, N, k, torch.from_numpy(np.ascontiguousarray(V0[y0 * N:y1 * N])),
                          degree=8, sweeps=3, bounds=O.csr_gershgorin(rp, ci, va), lines=lines)
    out[rank] = (r.values.numpy(), r.X.numpy(), r.res.numpy(), (y0 * N, y1 * N))
    dist.barrier()
    dist.destroy_process_group()


def _run(worker, world):
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    return dict(out)


def _same_up_to_sign(X, Y, tol):
    for j in range(X.shape[1]):
        assert min(np.abs(X[:, j] - Y[:, j]).max(), np.abs(X[:, j] + Y[:, j]).max()) < tol, j


@pytest.mark.parametrize("world", [2, 1])
def test_sharded_svd_matches_single_rank_oracle(world):
    from oracle import ofrr as O
    out = _run(_svd_worker, world)
    m, n, b, k = 600, 200, 16, 8
    A = wl.dense_svd(m, n, wl.config2_sigma(n), 5100)
    Amul, Atmul = O.dense_apply(A)
    ref = O.solve_svd(Amul, Atmul, m, n, k, wl.uniform_block(n, b, 5101), degree=2, max_sweeps=3, tol=0.0)
    U = np.zeros((m, k))
    for rank in range(world):
        s, V, Ur, res, (s0, s1) = out[rank]
        assert np.allclose(s, ref.values, rtol=1e-12, atol=0)
        assert np.allclose(res, ref.res, rtol=1e-6, atol=1e-15)
        _same_up_to_sign(V, ref.X, 1e-9)
        U[s0:s1] = Ur
    _same_up_to_sign(U, ref.U, 1e-9)


@pytest.mark.parametrize("world", [2])
def test_sharded_csr_eig_matches_single_rank_oracle(world):
    from oracle import ofrr as O
    out = _run(_eig_worker, world)
    N, b, k = 24, 12, 6
    rp, ci, va, _ = wl.grid_schrodinger_csr(N, 10.0, 5200)
    ref = O.solve_eig(O.csr_apply(rp, ci, va), N * N, k, wl.uniform_block(N * N, b, 5201), which="smallest",
                      filter="chebyshev", degree=8, max_sweeps=3, tol=0.0, bounds=O.csr_gershgorin(rp, ci, va))
    X = np.zeros((N * N, k))
    for rank in range(world):
        th, Xr, res, (r0, r1) = out[rank]
        assert np.allclose(th, ref.values, rtol=1e-12, atol=0)
        assert np.allclose(res, ref.res, rtol=1e-6, atol=1e-15)
        X[r0:r1] = Xr
    _same_up_to_sign(X, ref.X, 1e-9)


def test_partitions():
    from paper_2505_00281_gb300 import sharded as S
    assert S.row_partition(600, 2) == [(0, 304), (304, 600)]
    assert S.row_partition(10, 4) == [(0, 8), (8, 10), (10, 10), (10, 10)]
    assert S.grid_partition(24, 2) == [(0, 12), (12, 24)]
