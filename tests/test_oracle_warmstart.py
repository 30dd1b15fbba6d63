"""Pins of the learned-warm-start oracle (CPU only): the convolution against scipy's
correlation, every gradient against central finite differences, the Procrustes loss
against its closed form on a rotated copy, and Adam's first step against its formula."""
import numpy as np
import pytest
from scipy.signal import correlate

import workloads as wl
from oracle import warmstart as W


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 7, 9))
    Wt = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = W.conv3x3(x, Wt, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate(x[n, c], Wt[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)


def _num_grad(f, a, eps=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        old = a[i]
        a[i] = old + eps
        fp = f()
        a[i] = old - eps
        fm = f()
        a[i] = old
        g[i] = (fp - fm) / (2 * eps)
    return g


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    params = [(rng.standard_normal((3, 1, 3, 3)) * 0.5, rng.standard_normal(3) * 0.1),
              (rng.standard_normal((2, 3, 3, 3)) * 0.5, rng.standard_normal(2) * 0.1)]
    x = rng.standard_normal((1, 1, 5, 6))
    target = rng.standard_normal((1, 2, 5, 6))

    def loss():
        out = W.net_forward(params, x)[-1]
        return 0.5 * float(np.sum((out - target) ** 2))

    acts = W.net_forward(params, x)
    grads = W.net_backward(params, acts, acts[-1] - target)
    for (Wl, bl), (dW, db) in zip(params, grads):
        assert np.allclose(dW, _num_grad(loss, Wl), rtol=1e-5, atol=1e-7)
        assert np.allclose(db, _num_grad(loss, bl), rtol=1e-5, atol=1e-7)


def test_procrustes_loss_closed_form_and_gradient():
    rng = np.random.default_rng(3)
    Vs, _ = np.linalg.qr(rng.standard_normal((40, 5)))
    Q, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    L, g = W.procrustes_loss(Vs @ Q, Vs)                # an exact rotation: zero loss
    assert L < 1e-24 and np.abs(g).max() < 1e-12
    V = Vs @ Q * 0.7 + 0.01 * rng.standard_normal((40, 5))
    L, g = W.procrustes_loss(V, Vs)
    gn = _num_grad(lambda: W.procrustes_loss(V, Vs)[0], V)
    assert np.allclose(g, gn, rtol=1e-5, atol=1e-8)


def test_adam_first_step_is_a_signed_lr_step():
    p, g = np.array([1.0, -2.0, 3.0]), np.array([0.5, -0.1, 4.0])
    p1, m, v = W.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-7)   # bias-corrected m/sqrt(v) = sign(g)


def test_adam_steps_two_and_three_hand_expanded():
    """Adam past the first step, against moments expanded by hand.
    Gradients g1 = 1, g2 = 3, g3 = -2 on one parameter, b1 = 0.9, b2 = 0.999:
      m1 = 0.1,  v1 = 0.001
      m2 = 0.9 m1 + 0.1 * 3 = 0.39,      v2 = 0.999 v1 + 0.001 * 9 = 0.009999
      m3 = 0.9 m2 + 0.1 * (-2) = 0.151,  v3 = 0.999 v2 + 0.001 * 4 = 0.013989001
    bias corrections 1 - 0.9^2 = 0.19, 1 - 0.999^2 = 0.001999,
                     1 - 0.9^3 = 0.271, 1 - 0.999^3 = 0.002997001."""
    lr, eps = 0.01, 1e-8
    p, m, v = np.array([1.0]), np.zeros(1), np.zeros(1)
    p, m, v = W.adam_step(p, np.array([1.0]), m, v, 1, lr=lr)
    assert np.allclose([m[0], v[0]], [0.1, 0.001], rtol=1e-14)
    p1 = p.copy()
    p, m, v = W.adam_step(p, np.array([3.0]), m, v, 2, lr=lr)
    assert np.allclose([m[0], v[0]], [0.39, 0.009999], rtol=1e-14)
    step2 = lr * (0.39 / 0.19) / (np.sqrt(0.009999 / 0.001999) + eps)
    assert np.allclose(p, p1 - step2, rtol=1e-14)
    p2 = p.copy()
    p, m, v = W.adam_step(p, np.array([-2.0]), m, v, 3, lr=lr)
    assert np.allclose([m[0], v[0]], [0.151, 0.013989001], rtol=1e-14)
    step3 = lr * (0.151 / 0.271) / (np.sqrt(0.013989001 / 0.002997001) + eps)
    assert np.allclose(p, p2 - step3, rtol=1e-14)


def test_adam_constant_gradient_steps_are_signed_lr():
    """With the same gradient g at every step, m_t = g (1 - b1^t) and
    v_t = g^2 (1 - b2^t), so the bias-corrected step is lr sign(g) at every t
    (a wrong power in either correction breaks this at t >= 2)."""
    g = np.array([0.5, -0.1, 4.0])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        pn, m, v = W.adam_step(p, g, m, v, t, lr=0.01)
        assert np.allclose(m, g * (1 - 0.9 ** t), rtol=1e-13)
        assert np.allclose(v, g * g * (1 - 0.999 ** t), rtol=1e-13)
        assert np.allclose(pn - p, -0.01 * np.sign(g), rtol=1e-6)
        p = pn


def test_gaussian_potential_recipe():
    v = wl.gaussian_potential(64, 5)
    assert v.shape == (64, 64) and v.min() >= 0.0 and v.max() <= 8 * 20.0
    assert not np.array_equal(v, wl.gaussian_potential(64, 6))


def test_free_modes_are_laplacian_eigenvectors():
    """The network's input modes (package host logic): at scale 1/N orthonormal,
    and eigenvectors of the 5-point Dirichlet Laplacian with eigenvalues
    4 - 2 cos(p pi/(N+1)) - 2 cos(q pi/(N+1)), the k lowest in order."""
    from paper_2505_00281_gb300.warmstart import free_modes, layer_shapes
    from oracle import ofrr as O
    N, k = 20, 12
    V = free_modes(N, k).reshape(k, N * N).T.astype(np.float64) / N
    assert np.abs(V.T @ V - np.eye(k)).max() < 1e-6
    rp, ci, va = wl.grid_potential_csr(N, np.zeros(N * N))
    AV = O.csr_apply(rp, ci, va)(V)
    lam = np.sum(V * AV, axis=0)
    assert np.abs(AV - V * lam).max() < 1e-5
    t = np.arange(1, 2 * k) * np.pi / (N + 1)
    allv = np.sort((4 - 2 * np.cos(t)[:, None] - 2 * np.cos(t)[None, :]).ravel())
    assert np.allclose(lam, allv[:k], atol=1e-5)
    assert layer_shapes(16, 24, 3) == [(17, 24), (24, 24), (24, 16)]
