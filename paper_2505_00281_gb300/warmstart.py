"""Learned warm start: a convolutional network proposes the start block of Alg. 1.

The paper starts the subspace iteration from a random block (Alg. 1 draws V
from U(0,1)).  For a parameterised operator family, H(p) = -Lap + V_p on an
N x N grid (5-point Laplacian, Dirichlet boundary, row index y*N + x), a small
fully convolutional network maps the potential to the k wanted directions:

- input (1 + k channels): V_p / 20 and the k lowest Dirichlet modes of the
  free Laplacian, phi_pq(y, x) = (2N / (N + 1)) sin(pi p (y+1)/(N+1)) sin(pi q (x+1)/(N+1));
- layers: 3x3 convolutions with ReLU between them, the last one linear and
  added to the free modes (a skip connection: the network predicts how the
  potential bends the free modes);
- output (k channels) times 1/N: column c of the start block is channel c in
  row-major grid order (unit-norm columns for the free modes);
- loss: min over orthogonal R of |V R - V*|_F^2 against the converged Ritz
  vectors V* of the same operator (invariant to the order, signs and any
  rotation of degenerate eigenvectors);
- Adam on all parameters.

Every step runs in librr.so kernels (convolutions, ReLU masks, the Procrustes
gradient and its projected SVD, Adam); tensors here are device memory only.
A start block is the k network columns followed by random U(0,1) columns up
to the block size; the random block remains the fallback when no trained
network is given.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api
from ._lib import RR

__all__ = ["free_modes", "layer_shapes", "StartBlockNet", "eigen_targets", "train", "evaluate"]

POTENTIAL_SCALE = 1.0 / 20.0


def free_modes(N: int, k: int) -> np.ndarray:
    """The k lowest Dirichlet modes of the N x N 5-point Laplacian (ordered by
    p^2 + q^2, then p), as (k, N, N) FP32 images of amplitude 2N / (N + 1)."""
    pq = sorted(((p, q) for p in range(1, k + 2) for q in range(1, k + 2)), key=lambda t: (t[0] ** 2 + t[1] ** 2, t[0]))
    t = np.arange(1, N + 1, dtype=np.float64) * np.pi / (N + 1)
    amp = 2.0 * N / (N + 1)
    return np.stack([amp * np.outer(np.sin(p * t), np.sin(q * t)) for p, q in pq[:k]]).astype(np.float32)


def layer_shapes(k: int, hidden: int, depth: int):
    """(cin, cout) of each convolution: 1 + k -> hidden -> ... -> k."""
    assert depth >= 2
    return [(1 + k, hidden)] + [(hidden, hidden)] * (depth - 2) + [(hidden, k)]


class StartBlockNet:
    """Network, its gradients and Adam state in three flat FP32 device buffers."""

    def __init__(self, N: int, k: int, params, device="cuda"):
        self.N, self.k, self.device = N, k, device
        self.scale = 1.0 / N
        sizes = [(W.size, b.size) for W, b in params]
        total = sum(a + c for a, c in sizes)
        self.flat = torch.empty(total, dtype=torch.float32, device=device)
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.t = 0
        self.W, self.b, self.dW, self.db = [], [], [], []
        off = 0
        host = np.concatenate([np.concatenate([np.ravel(W), np.ravel(b)]) for W, b in params]).astype(np.float32)
        self.flat.copy_(torch.from_numpy(host))
        for (W, b) in params:
            for buf, dst in ((self.flat, self.W), (self.grad, self.dW)):
                dst.append(buf[off:off + W.size].view(W.shape))
            off += W.size
            for buf, dst in ((self.flat, self.b), (self.grad, self.db)):
                dst.append(buf[off:off + b.size])
            off += b.size
        self.x = torch.empty(1, 1 + k, N, N, dtype=torch.float32, device=device)
        self.x[0, 1:].copy_(torch.from_numpy(free_modes(N, k)))
        eye = torch.eye(k, dtype=torch.float64, device=device)
        self._eye = api.fortran(eye)

    def params(self):
        """Current parameters as host FP32 arrays [(W, b), ...]."""
        return [(W.detach().cpu().numpy().copy(), b.detach().cpu().numpy().copy()) for W, b in zip(self.W, self.b)]

    def set_potential(self, pot: torch.Tensor):
        """pot: (N, N) FP32 device tensor of V_p, already times POTENTIAL_SCALE."""
        self.x[0, 0].copy_(pot)

    def forward(self):
        acts = [self.x]
        h = self.x
        last = len(self.W) - 1
        for li, (W, b) in enumerate(zip(self.W, self.b)):
            add = self.x[:, 1:] if li == last else None
            h = api.rr_conv3x3_forward(h, W, b, relu=li < last, add=add)
            acts.append(h)
        return acts

    def loss_grad(self, out: torch.Tensor, Vstar: torch.Tensor):
        """Procrustes loss of V = scale * out against V* (n x k FP64, column-major)
        and its gradient with respect to `out`.  Returns (loss tensor[1], grad)."""
        n = self.N * self.N
        Vm = out.view(self.k, n).t()                       # n x k, column-major view
        M = api.rr_gram(Vm, Vstar)                         # (out)^T V*: same rotation as (scale out)^T V*
        _, U, Wm, _ = api.rr_pencil_svd(M, self._eye, self._eye)
        return api.rr_procrustes_grad(out, Vstar, U, Wm, self.scale)[::-1]

    def backward(self, acts, gout):
        g = gout
        for li in range(len(self.W) - 1, -1, -1):
            if li < len(self.W) - 1:
                api.rr_relu_mask(g, acts[li + 1])
            g = api.rr_conv3x3_backward(acts[li], self.W[li], g, self.dW[li], self.db[li], need_dx=li > 0)

    def adam(self, lr: float):
        self.t += 1
        api.rr_adam(self.flat, self.grad, self.m, self.v, self.t, lr)

    def propose(self, V0: torch.Tensor):
        """Overwrite the first k columns of the start block V0 (n x b FP64, column-major)."""
        out = self.forward()[-1]
        api.rr_net_block(out[0], self.scale, V0)
        return V0


def _params(k, block, degree, tol, v0, basis, phase1, max_sweeps):
    return api.make_params(k, block, degree, max_sweeps, tol, basis=basis, v0=v0, filter=RR.CHEBYSHEV,
                           which=RR.SMALLEST, refine=True, phase1_sweeps=phase1)


def eigen_targets(problems, k, block, degree, tol=1e-6, basis="bf16", phase1=1, max_sweeps=60):
    """Ritz vectors of each problem from random starts, to residual `tol` (the
    targets need not be more accurate than the network can be): a list of
    (potential (N, N) FP32 device, V* (n x k FP64), sweeps).  `problems` yields
    (potential (N, N) host FP64, CSR row_ptr / col_idx / values, V0 (n x block) host FP64)."""
    out = []
    for pot, rp, ci, va, V0 in problems:
        d = [torch.from_numpy(a).to("cuda") for a in (rp, ci, va)]
        v0 = api.fortran(torch.from_numpy(V0).to("cuda"))
        p = _params(k, block, degree, tol, v0, basis, phase1, max_sweeps)
        _, X, info = api.rr_eig(api.csr_operator(*d), p, pot.size)
        P = torch.from_numpy((pot * POTENTIAL_SCALE).astype(np.float32)).to("cuda")
        out.append((P, X, info["sweeps"]))
    return out


def train(net: StartBlockNet, data, epochs: int, lr: float, batch: int = 8, log=None, seed: int = 0):
    """Mini-batch Adam over the (potential, V*) pairs; returns the mean loss per epoch."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(data))
        tot = torch.zeros(1, dtype=torch.float64, device=net.device)
        for s0 in range(0, len(order), batch):
            net.grad.zero_()
            for i in order[s0:s0 + batch]:
                P, Vs = data[i][0], data[i][1]
                net.set_potential(P)
                acts = net.forward()
                loss, g = net.loss_grad(acts[-1], Vs)
                net.backward(acts, g)
                tot += loss
            net.adam(lr)
        hist.append(float(tot.item()) / len(data))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.4f}")
    return hist


ARMS = ("random", "modes", "learned")


def evaluate(net, problems, k, block, degree, tol=1e-10, basis="bf16", phase1=1, max_sweeps=60, arms=ARMS):
    """Solve each held-out problem from several start blocks and record sweeps,
    wall time (ms, the network's inference included) and the largest residual
    of the wanted pairs after each projection (Rayleigh-Ritz residuals):
      random:  U(0,1) (the paper's start);
      modes:   the `block` lowest free Dirichlet modes (no network);
      learned: the network's k columns, then the random start's columns k .. block - 1."""
    rows = []
    N = net.N
    modes = torch.from_numpy(free_modes(N, block)).to("cuda")
    for pot, rp, ci, va, V0 in problems:
        n = pot.size
        d = [torch.from_numpy(a).to("cuda") for a in (rp, ci, va)]
        op = api.csr_operator(*d)
        v_rand = api.fortran(torch.from_numpy(V0).to("cuda"))
        P = torch.from_numpy((pot * POTENTIAL_SCALE).astype(np.float32)).to("cuda")
        row = {}
        for name in arms:
            v0 = v_rand.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "modes":
                api.rr_net_block(modes, net.scale, v0)
            elif name == "learned":
                net.set_potential(P)
                net.propose(v0)
            p = _params(k, block, degree, tol, v0, basis, phase1, max_sweeps)
            _, _, info = api.rr_eig(op, p, n)
            torch.cuda.synchronize()
            row[name] = {"sweeps": info["sweeps"], "refine_sweeps": info["refine_sweeps"],
                         "n_converged": info["n_converged"], "ms": 1e3 * (time.perf_counter() - t0),
                         "res": info["res_history"][:info["sweeps"]]}
        rows.append(row)
    return rows
