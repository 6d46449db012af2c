"""Pins for the oracle's a-priori LES analysis (oracle/les.py).

The paper (Sec. 1, Sec. 2) names LES of the plume as the goal and a-priori
tests on the DNS database, but no filter or model; the reading is stated in
oracle/les.py.  Each pin is a closed form or an exact invariance:

* filter transfer function on single modes = the Dirichlet-kernel closed form
  sin(m k h) cot(k h / 2) / (2 m) per axis (mean preserved: G(0) = 1);
* a uniform velocity carries no sub-grid stress, whatever the density;
* a single shear mode u_x = A sin(k y) has tau_00 = A^2/2 (1 - G(2k) cos 2ky)
  - A^2 G(k)^2 sin^2 ky and no other component;
* the Favre stress is Galilean invariant (adding a uniform velocity to u
  leaves tau unchanged with a variable density);
* the Smagorinsky tensor of the filtered shear mode follows from the Gauss
  gradient's symbol.
"""
import numpy as np
import pytest

from oracle import les
from paper_1404_0959_gb300.inputs import random_fields, smooth_field


def grid(N):
    h = 2 * np.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return h, x, y, z


def dirichlet_G(k, h, m):
    th = k * h
    if abs(np.sin(th / 2)) < 1e-15:
        return 1.0
    return np.sin(m * th) / np.tan(th / 2) / (2 * m)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_filter_transfer_function_is_the_dirichlet_closed_form(m):
    N = 16
    h, x, y, z = grid(N)
    for kx, ky, kz in [(0, 0, 0), (1, 0, 0), (0, 3, 0), (0, 0, 5), (2, 1, 4), (8, 0, 0), (3, 7, 2)]:
        f = np.cos(kx * x + ky * y + kz * z + 0.3)
        want = dirichlet_G(kx, h, m) * dirichlet_G(ky, h, m) * dirichlet_G(kz, h, m) * f
        np.testing.assert_allclose(les.box_filter(f, m), want, atol=1e-13)
        assert abs(les.transfer(kx, h, m) - dirichlet_G(kx, h, m)) < 1e-13


def test_uniform_velocity_has_no_sgs_stress():
    N = 12
    rho = smooth_field(N, 3, 0.1, mean=1.0)
    u = [np.full((N, N, N), v) for v in (0.3, -0.2, 0.05)]
    _, _, tau = les.filtered_fields(rho, u, 2)
    for t in tau:
        assert np.max(np.abs(t)) < 1e-15


@pytest.mark.parametrize("m", [1, 2])
def test_single_shear_mode_stress_closed_form(m):
    N, A, k = 16, 0.7, 3
    h, x, y, z = grid(N)
    rho = np.ones((N, N, N))
    u = [A * np.sin(k * y), np.zeros_like(y), np.zeros_like(y)]
    rb, ut, tau = les.filtered_fields(rho, u, m)
    G1, G2 = dirichlet_G(k, h, m), dirichlet_G(2 * k, h, m)
    want00 = 0.5 * A * A * (1 - G2 * np.cos(2 * k * y)) - A * A * G1 * G1 * np.sin(k * y) ** 2
    np.testing.assert_allclose(tau[0], want00, atol=1e-14)
    for q in range(1, 6):
        assert np.max(np.abs(tau[q])) < 1e-15
    np.testing.assert_allclose(ut[0], A * G1 * np.sin(k * y), atol=1e-14)
    st = les.apriori(rho, u, h, m, 0.17)
    assert abs(st["k_sgs"] - 0.25 * A * A * (1 - G1 * G1)) < 1e-14


def test_favre_stress_is_galilean_invariant():
    N = 12
    rho, u, _, _ = random_fields(N, 0, False, seed=4, drho=0.1, noise=0.05)
    _, _, tau = les.filtered_fields(rho, u, 2)
    U = (0.8, -0.5, 0.3)
    _, _, tau2 = les.filtered_fields(rho, [u[i] + U[i] for i in range(3)], 2)
    for a, b in zip(tau, tau2):
        assert np.max(np.abs(a - b)) < 1e-13 * max(np.max(np.abs(a)), 1e-3)


def test_smagorinsky_tensor_of_a_shear_mode():
    N, A, k, m = 16, 0.4, 2, 1
    h, x, y, z = grid(N)
    rho = np.ones((N, N, N))
    u = [A * np.sin(k * y), np.zeros_like(y), np.zeros_like(y)]
    rb, ut, tau = les.filtered_fields(rho, u, m)
    S = les.strain(ut, h)
    # Gauss gradient symbol on sin(k y): d/dy -> kappa cos(k y)
    kappa = 2 * np.sin(k * h / 2) * (9 * np.cos(k * h / 2) - np.cos(3 * k * h / 2)) / (8 * h)
    S01 = 0.5 * A * dirichlet_G(k, h, m) * kappa * np.cos(k * y)
    np.testing.assert_allclose(S[1], S01, atol=1e-14)
    for q in (0, 2, 3, 4, 5):
        assert np.max(np.abs(S[q])) < 1e-14
    delta = 2 * m * h
    B = les.smagorinsky_tensor(rb, S, delta)
    np.testing.assert_allclose(B[1], -4 * delta * delta * np.abs(S01) * S01, atol=1e-14)
    st = les.apriori(rho, u, h, m, 0.2)
    # Pi_M = -Cs^2 <B_ij S_ij> = Cs^2 <8 Delta^2 |S01|^3> (two off-diagonal entries)
    assert abs(st["pi_model"] - 0.04 * 8 * delta * delta * np.mean(np.abs(S01) ** 3)) < 1e-14
