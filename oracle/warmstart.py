"""FP64 oracle of the learned warm start (the start-block network and its training step).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper starts its iteration from a random block (Alg. 1: V drawn U(0,1)); the
learned warm start replaces that start block by the output of a small fully
convolutional network of the operator's potential, trained on Ritz vectors the
plain method produced.  Everything here is the plain definition, in FP64:

- conv3x3: zero-padded 3x3 cross-correlation, NCHW, weights (cout, cin, 3, 3),
  one bias per output channel;  y[n,o,i,j] = b[o] + sum_{c,dy,dx} W[o,c,dy,dx] x[n,c,i+dy-1,j+dx-1];
- ReLU between layers, none after the last;
- the network output (one image, C channels) read as the n x C start block whose
  column c is channel c flattened in row-major grid order, times a fixed scale;
- the Procrustes-aligned squared error against the reference Ritz vectors V* (n x C,
  orthonormal): L = min_{R orthogonal} |V R - V*|_F^2, R = U W^T from the SVD
  V^T V* = U S W^T, so L = |V|_F^2 - 2 trace(S) + |V*|_F^2 and dL/dV = 2 (V R - V*) R^T;
- Adam (bias-corrected first and second moments).
"""
from __future__ import annotations

import numpy as np

__all__ = ["conv3x3", "conv3x3_backward", "relu", "net_forward", "net_backward",
           "procrustes_loss", "adam_step"]


def conv3x3(x, W, b):
    """x (N, C, H, Wd), W (O, C, 3, 3), b (O,) -> (N, O, H, Wd), zero padding."""
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    y = np.zeros((N, W.shape[0], H, Wd)) + np.asarray(b, np.float64)[None, :, None, None]
    for dy in range(3):
        for dx in range(3):
            patch = xp[:, :, dy:dy + H, dx:dx + Wd]          # x[n, c, i + dy - 1, j + dx - 1]
            y += np.einsum("oc,nchw->nohw", W[:, :, dy, dx], patch)
    return y


def conv3x3_backward(x, W, dy):
    """Gradients of conv3x3 for upstream dy (N, O, H, Wd): (dx, dW, db)."""
    x = np.asarray(x, np.float64)
    W = np.asarray(W, np.float64)
    dy = np.asarray(dy, np.float64)
    N, C, H, Wd = x.shape
    xp = np.zeros((N, C, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + H, kx:kx + Wd]
            dW[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, patch)
            dxp[:, :, ky:ky + H, kx:kx + Wd] += np.einsum("oc,nohw->nchw", W[:, :, ky, kx], dy)
    return dxp[:, :, 1:H + 1, 1:Wd + 1], dW, dy.sum(axis=(0, 2, 3))


def relu(z):
    return np.maximum(z, 0.0)


def net_forward(params, x):
    """params = [(W, b), ...]; returns the list of layer inputs and the output."""
    acts = [np.asarray(x, np.float64)]
    h = acts[0]
    for li, (W, b) in enumerate(params):
        z = conv3x3(h, W, b)
        h = relu(z) if li + 1 < len(params) else z
        acts.append(h)
    return acts


def net_backward(params, acts, dout):
    """Gradients [(dW, db), ...] of the loss for d(loss)/d(output) = dout."""
    grads = [None] * len(params)
    g = np.asarray(dout, np.float64)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li + 1 < len(params):
            g = g * (acts[li + 1] > 0)                       # through the ReLU of layer li
        dx, dW, db = conv3x3_backward(acts[li], W, g)
        grads[li] = (dW, db)
        g = dx
    return grads


def procrustes_loss(V, Vstar):
    """L = min_R |V R - V*|^2 (R orthogonal) and dL/dV."""
    V = np.asarray(V, np.float64)
    Vstar = np.asarray(Vstar, np.float64)
    U, S, Wt = np.linalg.svd(V.T @ Vstar)
    R = U @ Wt
    L = float(np.sum((V @ R - Vstar) ** 2))
    return L, 2.0 * (V @ R - Vstar) @ R.T


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t = step count starting at 1); returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
