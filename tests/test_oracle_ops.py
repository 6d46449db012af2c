"""Pins for the oracle's stencils: closed-form Fourier symbols and measured order.

Sec. 2 of the paper specifies "fourth order central interpolation"; the
symbols below follow from the stencil definitions by elementary
trigonometry (a sampled mode e^{ikx} is an eigenfunction of every
shift-invariant stencil on the periodic grid), not from the oracle code.
"""
import math

import numpy as np
import pytest

from oracle import ops


def mode_1d(N, k, d):
    """e^{i k x} sampled at cell centres along direction d, constant elsewhere."""
    h = 2 * math.pi / N
    x = (np.arange(N) + 0.5) * h
    shape = [1, 1, 1]
    shape[ops.axis(d)] = N
    return np.exp(1j * k * x).reshape(shape), x, h


def face_mode(N, k, d):
    h = 2 * math.pi / N
    xf = (np.arange(N) + 1.0) * h
    shape = [1, 1, 1]
    shape[ops.axis(d)] = N
    return np.exp(1j * k * xf).reshape(shape)


@pytest.mark.parametrize("d", [0, 1, 2])
@pytest.mark.parametrize("N,k", [(16, 1), (16, 5), (24, 7), (32, 3)])
def test_symbols(N, k, d):
    f, x, h = mode_1d(N, k, d)
    ef = face_mode(N, k, d)
    th = k * h / 2
    sym_I4 = (9 * np.cos(th) - np.cos(3 * th)) / 8
    sym_G4 = 1j * (27 * np.sin(th) - np.sin(3 * th)) / (12 * h)
    sym_G2 = 2j * np.sin(th) / h
    sym_Gc = 1j * (10 * np.sin(k * h) - np.sin(2 * k * h)) / (8 * h)
    sym_D = 2j * np.sin(th) / h
    np.testing.assert_allclose(ops.I4(f, d), sym_I4 * ef, rtol=0, atol=1e-14)
    np.testing.assert_allclose(ops.G4(f, d, h), sym_G4 * ef, rtol=0, atol=1e-12 * k)
    np.testing.assert_allclose(ops.G2(f, d, h), sym_G2 * ef, rtol=0, atol=1e-12 * k)
    np.testing.assert_allclose(ops.Gc(f, d, h), sym_Gc * f, rtol=0, atol=1e-12 * k)
    np.testing.assert_allclose(ops.Dd(ef, d, h), sym_D * f, rtol=0, atol=1e-12 * k)
    # D o G4 (viscous second derivative) symbol, closed form
    sym_DG4 = -(2 * np.sin(th) / h) * (54 * np.sin(th) - 2 * np.sin(3 * th)) / (24 * h)
    np.testing.assert_allclose(ops.Dd(ops.G4(f, d, h), d, h), sym_DG4 * f, rtol=0, atol=1e-11 * k * k)


def _order(op, exact, Ns):
    errs = []
    for N in Ns:
        h = 2 * math.pi / N
        x = (np.arange(N) + 0.5) * h
        f = np.sin(x + 0.3).reshape(1, 1, N)
        errs.append(np.max(np.abs(op(f, h) - exact(x, h).reshape(1, 1, N))))
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)], errs


def test_order_I4():
    orders, errs = _order(lambda f, h: ops.I4(f, 0), lambda x, h: np.sin(x + h / 2 + 0.3), [16, 32, 64, 128])
    assert all(abs(o - 4.0) < 0.1 for o in orders), orders
    # leading error constant 3/128 (kh)^4 relative to the amplitude
    h = 2 * math.pi / 128
    assert abs(errs[-1] / (3 / 128 * h ** 4) - 1) < 0.01


def test_order_G4():
    orders, _ = _order(lambda f, h: ops.G4(f, 0, h), lambda x, h: np.cos(x + h / 2 + 0.3), [16, 32, 64, 128])
    assert all(abs(o - 4.0) < 0.1 for o in orders), orders


def test_order_Gc_is_two():
    # Gauss gradient built on I4 face values is second order: error k^3 h^2 / 24
    orders, errs = _order(lambda f, h: ops.Gc(f, 0, h), lambda x, h: np.cos(x + 0.3), [32, 64, 128, 256])
    assert all(abs(o - 2.0) < 0.05 for o in orders), orders
    h = 2 * math.pi / 256
    assert abs(errs[-1] / (h ** 2 / 24) - 1) < 0.01


def _plane_wave(N, kvec, amp):
    h = 2 * math.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ph = np.exp(1j * (kvec[0] * x + kvec[1] * y + kvec[2] * z))
    return [a * ph for a in amp], ph, h


def _g(k, h):
    return (10 * np.sin(k * h) - np.sin(2 * k * h)) / (8 * h)


def _s(k, h):
    th = k * h / 2
    return (2 * np.sin(th) / h) * (27 * np.sin(th) - np.sin(3 * th)) / (12 * h)


def test_viscous_stress_closed_form():
    """D tau for a plane wave: mu[-(sum_d s_d) a_m - g_m (g.a)/3].

    Follows from tau_dm = mu(du_m/dx_d + du_d/dx_m - 2/3 delta div u) with the
    discrete symbols; a transposed gradient or a wrong 2/3 changes it.
    """
    N, mu = 16, 0.37
    kvec = (1, -2, 3)
    amp = (0.3, -0.7, 0.45)
    u, ph, h = _plane_wave(N, kvec, amp)
    visc = ops.div_stress(u, mu, h)
    g = [_g(k, h) for k in kvec]
    ssum = sum(_s(k, h) for k in kvec)
    gdota = sum(g[l] * amp[l] for l in range(3))
    for m in range(3):
        expect = mu * (-ssum * amp[m] - g[m] * gdota / 3.0) * ph
        np.testing.assert_allclose(visc[m], expect, rtol=0, atol=1e-12)


def test_convection_closed_form():
    """Uniform flux phi = U: L_m = -i (U.g) a_m + (D tau)_m."""
    N, mu = 16, 0.0
    kvec = (2, 1, -1)
    amp = (0.1, 0.2, -0.3)
    U = (0.4, -0.25, 0.6)
    u, ph, h = _plane_wave(N, kvec, amp)
    phi = [np.full((N, N, N), U[d], dtype=complex) for d in range(3)]
    out = ops.L(u, phi, mu, h)
    g = [_g(k, h) for k in kvec]
    udotg = sum(U[d] * g[d] for d in range(3))
    for m in range(3):
        np.testing.assert_allclose(out[m], -1j * udotg * amp[m] * ph, rtol=0, atol=1e-13)
