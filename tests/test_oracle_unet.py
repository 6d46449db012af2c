"""Pins for the oracle U-Net: brute-force convolution, finite-difference
gradients of every layer, translation equivariance, Adam's first step."""
import numpy as np
import pytest

from oracle import unet


def brute_conv(x, W, b, stride=1):
    C, N = x.shape[0], x.shape[1]
    cout = W.shape[2]
    No = N // stride
    y = np.zeros((cout, No, No, No))
    for co in range(cout):
        for k in range(No):
            for j in range(No):
                for i in range(No):
                    s = b[co]
                    for ti, (dz, dy, dx) in enumerate(unet.TAPS):
                        for ci in range(C):
                            s += W[ti, ci, co] * x[ci, (stride * k + dz) % N, (stride * j + dy) % N,
                                                   (stride * i + dx) % N]
                    y[co, k, j, i] = s
    return y


@pytest.mark.parametrize("stride", [1, 2])
def test_conv_matches_brute_force(stride):
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 4, 4, 4))
    W = rng.standard_normal((27, 2, 3))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(unet.conv(x, W, b, stride), brute_conv(x, W, b, stride), rtol=1e-12, atol=1e-12)


def _loss(P, x, R):
    y, _ = unet.forward(P, x)
    return float(np.sum(y * R))


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    N = 8
    x = rng.standard_normal((2, N, N, N))
    P = unet.init_params(2, seed=2)
    R = rng.standard_normal((1, N, N, N))
    y, cache = unet.forward(P, x)
    G, dx = unet.backward(P, cache, R)
    eps = 1e-6
    for name in P:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = _loss(P, x, R)
            flat[idx] = old - eps
            lm = _loss(P, x, R)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)
    xf = x.reshape(-1)
    for idx in rng.choice(xf.size, size=6, replace=False):
        old = xf[idx]
        xf[idx] = old + eps
        lp = _loss(P, x, R)
        xf[idx] = old - eps
        lm = _loss(P, x, R)
        xf[idx] = old
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - dx.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_translation_equivariance_by_four_cells():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 8, 8, 8))
    P = unet.init_params(2, seed=4)
    y, _ = unet.forward(P, x)
    ys, _ = unet.forward(P, np.roll(x, 4, axis=3))
    np.testing.assert_allclose(np.roll(y, 4, axis=3), ys, rtol=1e-12, atol=1e-12)


def test_loss_gradient_and_adam_first_step():
    rng = np.random.default_rng(5)
    y = rng.standard_normal((1, 4, 4, 4))
    t = rng.standard_normal((1, 4, 4, 4))
    L, g = unet.loss_rel_mse(y, t)
    assert abs(L - np.sum((y - t) ** 2) / np.sum(t * t)) < 1e-15
    eps = 1e-7
    y2 = y.copy()
    y2[0, 1, 2, 3] += eps
    assert abs((unet.loss_rel_mse(y2, t)[0] - L) / eps - g[0, 1, 2, 3]) < 1e-6
    p = rng.standard_normal(5)
    gr = rng.standard_normal(5)
    p1, m, v = unet.adam_update(p, gr, np.zeros(5), np.zeros(5), 1, 1e-3)
    # first Adam step moves each parameter by lr * g / (|g| + eps)
    np.testing.assert_allclose(p1, p - 1e-3 * gr / (np.abs(gr) + 1e-8), rtol=1e-12)
