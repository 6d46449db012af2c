"""Pins for the oracle's turbulence diagnostics (closed forms, Parseval)."""
import math

import numpy as np

from oracle import diag, ic


def grid(N):
    h = 2 * math.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z, h


def g1(h):
    return (10 * np.sin(h) - np.sin(2 * h)) / (8 * h)


def test_taylor_green_closed_forms():
    """TG: u = A(sin x cos y cos z, -cos x sin y cos z, 0).

    <u^2> = <v^2> = A^2/8, so KE_u = A^2/8; curl gives omega_z = 2A sin x sin y
    cos z and |omega|^2 mean 6 A^2/8 times g^2 (one discrete derivative per
    component), so enstrophy = 3 A^2 g^2 / 8; microscale^2 = 1/g^2.
    """
    N, A = 16, 0.3
    x, y, z, h = grid(N)
    u = [A * np.sin(x) * np.cos(y) * np.cos(z), -A * np.cos(x) * np.sin(y) * np.cos(z), 0 * x]
    rho = 1.0 + 0.1 * np.sin(x)
    d = diag.diagnostics(rho, u, h, nbins=N)
    g = g1(h)
    assert abs(d["ke_u"] - A * A / 8) < 1e-15
    assert abs(d["enstrophy"] - 3 * A * A * g * g / 8) < 1e-14
    assert abs(d["taylor"] - 1 / g) < 1e-13
    assert abs(d["rho_rms"] - 0.1 / math.sqrt(2)) < 1e-15
    # TG lives in shell round(sqrt(3)) = 2
    assert abs(d["spectrum"][2] - A * A / 8) < 1e-15
    assert abs(d["spectrum"].sum() - A * A / 8) < 1e-15


def test_single_mode_shell_and_mass_weighting():
    N, A = 12, 0.5
    x, y, z, h = grid(N)
    u = [0 * x, A * np.cos(3 * x), 0 * x]
    rho = np.full_like(x, 2.0)
    d = diag.diagnostics(rho, u, h, nbins=8)
    assert abs(d["ke_u"] - A * A / 4) < 1e-15
    assert abs(d["ke"] - 2 * A * A / 4) < 1e-15
    e = d["spectrum"]
    assert abs(e[3] - A * A / 4) < 1e-15
    assert np.all(np.abs(np.delete(e, 3)) < 1e-30)


def test_parseval_random_field():
    N = 16
    u = ic.spectral_velocity(N, 3.0, 0.4, 5)
    h = 2 * math.pi / N
    nb = int(math.ceil(math.sqrt(3) * N / 2)) + 1
    d = diag.diagnostics(np.ones_like(u[0]), u, h, nbins=nb)
    assert abs(d["spectrum"].sum() - d["ke_u"]) < 1e-14
    assert abs(d["ke_u"] - 0.5 * 0.4 ** 2) < 1e-14


def test_q_criterion_solid_rotation_and_strain():
    """u = (sin y, -sin x, 0): du/dy = g cos y, dv/dx = -g cos x (g the discrete
    gradient symbol), so Omega_xy = g (cos y + cos x)/2, S_xy = g (cos y - cos x)/2
    and Q = (|Omega|^2 - |S|^2)/2 = g^2 cos x cos y: rotation-dominated (Q > 0)
    where cos x cos y > 0, strain-dominated elsewhere."""
    N = 16
    x, y, z, h = grid(N)
    u = [np.sin(y), -np.sin(x), 0 * x]
    q = diag.q_criterion(u, h)
    g = g1(h)
    np.testing.assert_allclose(q, g * g * np.cos(x) * np.cos(y), rtol=0, atol=1e-13)
