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


# ---- residual-form preconditioner definitions ---------------------------------------------


def _operator(N=8, seed=3):
    from oracle import piso
    from paper_1404_0959_gb300.inputs import smooth_field
    prm = piso.Params(N=N)
    psi = 1.0 + smooth_field(N, seed, 0.1)
    dt = 0.07
    matvec, _ = piso.helmholtz(prm, psi, dt)
    return prm, psi, dt, matvec


def test_jacobi_diag_and_weight_channel_are_the_operators_entries():
    """d is the diagonal entry of M (read off M applied to a unit vector), and the
    second input channel is six times the neighbour entry over the diagonal."""
    prm, psi, dt, matvec = _operator()
    N, h = prm.N, prm.h
    for c in [(0, 0, 0), (3, 5, 7), (7, 2, 1)]:
        e = np.zeros((N, N, N))
        e[c] = 1.0
        col = matvec(e)
        diag = col[c]
        nbr = col[c[0], c[1], (c[2] + 1) % N]
        assert abs(unet.jacobi_diag(psi, dt, h)[c] / diag - 1) < 1e-14
        w = unet.network_input(np.ones((N, N, N)), psi, dt, h)[1]
        assert abs(w[c] - 6.0 * (-nbr) / diag) < 1e-14
        assert 0.0 < w[c] < 1.0


def test_zero_last_layer_gives_the_jacobi_direction():
    prm, psi, dt, matvec = _operator()
    P = unet.init_params(2, seed=1)
    P["out.W"][:] = 0.0
    P["out.b"][:] = 0.0
    r = np.random.default_rng(4).standard_normal(psi.shape)
    z = unet.direction(P, r, psi, dt, prm.h)
    d = np.array([matvec(np.eye(1, psi.size, k).reshape(psi.shape)).reshape(-1)[k] for k in range(0, psi.size, 97)])
    np.testing.assert_allclose(z.reshape(-1)[::97], r.reshape(-1)[::97] / d, rtol=1e-13)


def test_target_direction_solves_the_system(monkeypatch):
    """With the network output replaced by the training target of a pair (r, e),
    M e = r, the direction is e itself: target and direction use one scaling."""
    from oracle import krylov
    prm, psi, dt, matvec = _operator()
    r = np.random.default_rng(5).standard_normal(psi.shape)
    e, _, _, _ = krylov.pcg(matvec, r, unet.jacobi_diag(psi, dt, prm.h), 1e-14, 500)
    t = unet.training_target(r, e, psi, dt, prm.h)
    monkeypatch.setattr(unet, "forward", lambda P, x: (t, None))
    z = unet.direction(None, r, psi, dt, prm.h)
    assert np.linalg.norm(matvec(z) - r) / np.linalg.norm(r) < 1e-12


def test_direction_scales_with_the_residual():
    prm, psi, dt, matvec = _operator()
    P = unet.init_params(2, seed=2)
    r = np.random.default_rng(6).standard_normal(psi.shape)
    z1 = unet.direction(P, r, psi, dt, prm.h)
    z2 = unet.direction(P, 3.5 * r, psi, dt, prm.h)
    np.testing.assert_allclose(z2, 3.5 * z1, rtol=1e-12, atol=1e-14 * np.abs(z1).max())
    np.testing.assert_allclose(unet.network_input(7.0 * r, psi, dt, prm.h), unet.network_input(r, psi, dt, prm.h),
                               rtol=1e-13)
    assert not np.any(unet.direction(P, 0.0 * r, psi, dt, prm.h))
