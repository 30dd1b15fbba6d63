"""Row-sharded schedule of the method across ranks (one process per GPU).

The data-parallel dimension of the path is the rows of the operator and of
the tall blocks: everything on the path is row-local except the pivot search
of Algorithm 8 and the projection products, which sum over rows.  Rank r
holds a contiguous range of rows of A (dense) or of grid lines (CSR) and the
same rows of every tall block; the schedule per projection is

  filter     dense SVD: W_r = A_r V (V replicated), all-gather W, U = Alg. 8(W)
             (replicated), Z = sum_r A_r^T U_r (all-reduce), V = Alg. 8(Z);
             CSR eigen: the Chebyshev steps on the local lines after a halo
             exchange of the neighbouring grid lines, all-gather, Alg. 8;
  projection the partial G / H (Alg. 3) or B, G_U (Alg. 5) of the local rows,
             one FP64 all-reduce (sum) of them packed together; G_V is
             replicated;
  solve      the small pencil, replicated on every rank (same input, same
             result);
  lift       the local rows of the Ritz vectors (U_r Y, V Z); the residual
             norms of the local rows, summed with one all-reduce.

The all-gather before Algorithm 8 replaces its per-column global pivot search
(one tiny collective per column) by one exchange of the block; the pivots and
the basis are those of the single-rank process, so the sharded method takes
the same steps as the single-rank one, up to the order of the summed
products.

Local compute goes through an ``ops`` object (the product kernels on a GPU;
any implementation with the same operations elsewhere), communication through
``torch.distributed``; tensors are torch tensors on the ops' device.  The
operations ``ops`` must provide are listed in ``LocalOps``.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Protocol

import torch
import torch.distributed as dist

__all__ = ["LocalOps", "row_partition", "grid_partition", "local_csr", "svd_sharded", "eig_csr_sharded",
           "ShardedResult"]


class LocalOps(Protocol):
    def mm(self, A, X): ...                 # A_r X (dense rows of A times a replicated block)
    def mm_t(self, A, X): ...               # A_r^T X_r (partial sum over this rank's rows)
    def spmm(self, csr, X_ext): ...         # local CSR rows times the halo-extended block
    def basis(self, W): ...                 # Algorithm 8 on a whole (gathered) block
    def colscale(self, W): ...              # column inf-norm scaling (Sec. 2)
    def gram(self, X, Y): ...               # X^T Y, FP64-accurate
    def pencil_svd(self, B, Gu, Gv): ...    # (s descending, Y, Z), U Y and V Z orthonormal
    def pencil_eig(self, H, G): ...         # (theta ascending, Y), Y^T G Y = I
    def colnorm2(self, R): ...              # squared 2-norms of the columns


def row_partition(n: int, world: int, align: int = 8):
    """Contiguous row ranges [(start, end)] for `world` ranks, boundaries on
    multiples of `align` rows (whole 16-byte vectors of the blocks)."""
    per = -(-n // world)
    per = -(-per // align) * align
    return [(min(n, r * per), min(n, (r + 1) * per)) for r in range(world)]


def grid_partition(N: int, world: int):
    """Grid lines [(y0, y1)] per rank for an N x N grid (rows y N .. y1 N)."""
    per = -(-N // world)
    return [(min(N, r * per), min(N, (r + 1) * per)) for r in range(world)]


@dataclass
class LocalCSR:
    row_ptr: torch.Tensor
    col_idx: torch.Tensor
    values: torch.Tensor
    halo_up: int     # grid lines before the local ones in the extended block (0 or 1)
    halo_down: int


def local_csr(row_ptr, col_idx, values, N: int, y0: int, y1: int) -> LocalCSR:
    """The CSR rows of grid lines [y0, y1) with columns renumbered into the
    extended block [line y0-1 (if any); lines y0..y1-1; line y1 (if any)]."""
    up = 1 if y0 > 0 else 0
    down = 1 if y1 < N else 0
    r0, r1 = y0 * N, y1 * N
    rp = row_ptr[r0:r1 + 1] - row_ptr[r0]
    lo, hi = int(row_ptr[r0]), int(row_ptr[r1])
    ci = col_idx[lo:hi] - (y0 - up) * N
    return LocalCSR(rp.clone(), ci.clone(), values[lo:hi].clone(), up, down)


@dataclass
class ShardedResult:
    values: torch.Tensor     # k wanted values (replicated)
    X: torch.Tensor          # local rows of the eigenvectors / right singular vectors (V: replicated)
    U: torch.Tensor | None   # local rows of the left singular vectors
    res: torch.Tensor        # residuals of the k wanted pairs (replicated)
    sweeps: int


def _all_gather_rows(X_local, counts):
    """Concatenate every rank's rows (ranks may hold different row counts)."""
    world = len(counts)
    b = X_local.shape[1]
    mx = max(counts)
    pad = torch.zeros(mx, b, dtype=X_local.dtype, device=X_local.device)
    pad[:X_local.shape[0]] = X_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def _allreduce(t):
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def svd_sharded(ops: LocalOps, A_r, m: int, n: int, k: int, V0, *, degree: int, sweeps: int,
                rows) -> ShardedResult:
    """Algorithm 1 / 5 / 8 for the largest singular triplets with A's rows
    sharded: A_r holds rows rows[rank] of the m x n operator; V0 (n x b) is
    the replicated start block.  Runs `sweeps` projections."""
    rank = dist.get_rank()
    counts = [e - s for s, e in rows]
    s0, s1 = rows[rank]
    V = ops.colscale(V0)
    b = V.shape[1]
    for _ in range(sweeps):
        for _ in range(degree):
            W = _all_gather_rows(ops.mm(A_r, V), counts)        # A V
            U = ops.basis(W)[s0:s1]                             # local rows of Alg. 8's basis
            V = ops.basis(_allreduce(ops.mm_t(A_r, U)))         # A^T U, summed over ranks
        P_r = ops.mm(A_r, V)
        # Algorithm 5's projected blocks: B and G_U summed over rows in one
        # all-reduce; G_V from the replicated V
        pk = torch.cat([ops.gram(U, P_r), ops.gram(U, U)], dim=1)
        _allreduce(pk)
        B, Gu = pk[:, :b], pk[:, b:]
        s, Y, Z = ops.pencil_svd(B, Gu, ops.gram(V, V))
        Ut_r = ops.mm(U, Y)                                    # local rows of U~ = U Y
        Vt = ops.mm(V, Z)                                      # V~ = V Z (replicated)
        # residuals of the k wanted triplets: |A v - s u|^2 row-local, summed;
        # A^T u summed over ranks
        R1 = ops.colnorm2(ops.mm(A_r, Vt[:, :k]) - Ut_r[:, :k] * s[:k])
        AtU = _allreduce(ops.mm_t(A_r, Ut_r[:, :k]))
        r2 = ops.colnorm2(AtU - Vt[:, :k] * s[:k])
        res = torch.sqrt(_allreduce(R1) + r2) / s[:k]
        V = Vt
    return ShardedResult(s[:k], Vt[:, :k], Ut_r[:, :k], res, sweeps)


def _halo(ops, csr: LocalCSR, Y_r, N: int):
    """Y_r extended by the neighbouring grid lines (point-to-point exchange)."""
    rank, world = dist.get_rank(), dist.get_world_size()
    b = Y_r.shape[1]
    parts = []
    reqs = []
    if csr.halo_up:
        up = torch.empty(N, b, dtype=Y_r.dtype, device=Y_r.device)
        reqs.append(dist.irecv(up, src=rank - 1))
        reqs.append(dist.isend(Y_r[:N].contiguous(), dst=rank - 1))
        parts.append(up)
    parts.append(Y_r)
    if csr.halo_down:
        down = torch.empty(N, b, dtype=Y_r.dtype, device=Y_r.device)
        reqs.append(dist.irecv(down, src=rank + 1))
        reqs.append(dist.isend(Y_r[-N:].contiguous(), dst=rank + 1))
        parts.append(down)
    for q in reqs:
        q.wait()
    return torch.cat(parts, dim=0)


def _apply(ops, csr, Y_r, N):
    return ops.spmm(csr, _halo(ops, csr, Y_r, N))


def eig_csr_sharded(ops: LocalOps, csr: LocalCSR, N: int, k: int, V0_r, *, degree: int, sweeps: int,
                    bounds, lines) -> ShardedResult:
    """Algorithm 1 / 3 / 8 for the lowest eigenpairs of a symmetric CSR grid
    operator with a degree-d scaled Chebyshev filter (the chebfsi filter cited
    in Sec. 2): rank r holds grid lines lines[rank] of the N x N grid and the
    same rows of every block (V0_r: its rows of the start block).  Interval
    rule as the single-rank solver: the first sweep damps
    [lo + 0.1 (up - lo), up] normalised at lo, later sweeps
    [max Ritz value, up] normalised at the min Ritz value."""
    rank = dist.get_rank()
    counts = [(e - s) * N for s, e in lines]
    r0 = lines[rank][0] * N
    r1 = r0 + counts[rank]
    lo, up = bounds
    V = ops.colscale(_all_gather_rows(V0_r, counts))[r0:r1]
    theta_all = None
    for _ in range(sweeps):
        a, a0 = (lo + 0.1 * (up - lo), lo) if theta_all is None else (float(theta_all.max()), float(theta_all.min()))
        e, c = (up - a) / 2.0, (up + a) / 2.0
        s1 = e / (a0 - c)
        Y0 = V
        Y1 = (s1 / e) * (_apply(ops, csr, Y0, N) - c * Y0)
        sj = s1
        for _ in range(2, degree + 1):
            sn = 1.0 / (2.0 / s1 - sj)
            Y2 = (2.0 * sn / e) * (_apply(ops, csr, Y1, N) - c * Y1) - (sj * sn) * Y0
            Y0, Y1, sj = Y1, Y2, sn
        V = ops.basis(_all_gather_rows(Y1, counts))[r0:r1]   # Alg. 8 on the gathered block
        AV = _apply(ops, csr, V, N)
        pk = torch.cat([ops.gram(V, AV), ops.gram(V, V)], dim=1)
        _allreduce(pk)
        b = V.shape[1]
        H, G = pk[:, :b], pk[:, b:]
        theta, Y = ops.pencil_eig(0.5 * (H + H.T), 0.5 * (G + G.T))
        X_r = ops.mm(V, Y)
        nrm = torch.sqrt(_allreduce(ops.colnorm2(X_r)))
        X_r = X_r / nrm
        theta_all = theta
        R = _apply(ops, csr, X_r[:, :k], N) - X_r[:, :k] * theta[:k]
        res = torch.sqrt(_allreduce(ops.colnorm2(R))) / theta[:k].abs()
        V = X_r
    return ShardedResult(theta[:k], X_r[:, :k], None, res, sweeps)
