"""Pins for the oracle's two-way coupled dusty gas (oracle/piso.py, coupling = TWO_WAY).

With the first-order particle velocity u_p = u - tau_p a (Sec. 2 par. 2) the drag per unit dust
mass is the gas acceleration a, so the gas feels f = -rho Ysum a and accelerates with the inertia
rho (1 + Ysum): Marble's dusty gas (the Sec. 2 par. 3 footnote's reference), which for a uniform
loading Y is an effective gas with sound speed c / sqrt(1 + Y) and kinematic viscosity
nu / (1 + Y).  The pins: an unloaded gas takes the one-way step bit for bit; the momentum the gas
gains over a step is exactly the trapezoidal impulse of the reaction force; the acoustic frequency
and the viscous decay rate of the effective gas, approached as dt -> 0.
"""
import math

import numpy as np
import pytest

from oracle import diag, ops, piso


def grid(N):
    h = 2 * math.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    return x, y, z, h


def loaded_state(prm, seed, Ymean=0.2):
    rng = np.random.default_rng(seed)
    sh = (prm.N,) * 3
    rho = 1.0 + 0.1 * rng.standard_normal(sh)
    u = [0.2 * rng.standard_normal(sh) for _ in range(3)]
    Y = [Ymean * (0.5 + rng.random(sh)) for _ in range(prm.n_dust)]
    return piso.make_state(prm, rho, u, Y)


def test_unloaded_two_way_is_one_way():
    """Ysum = 0: no reaction force and the gas inertia alone, bit for bit."""
    prm1 = piso.Params(N=8, tau_p=[0.05, 0.2], Y0=[0.0, 0.0], p_tol=1e-12)
    prm2 = piso.Params(N=8, tau_p=[0.05, 0.2], Y0=[0.0, 0.0], p_tol=1e-12, coupling=piso.TWO_WAY)
    st = loaded_state(prm1, 4)
    st["Y"] = [np.zeros_like(st["rho"]) for _ in range(2)]
    a, _ = piso.step(prm1, st, dt=0.02)
    b, _ = piso.step(prm2, st, dt=0.02)
    for key in ("rho", "p"):
        assert np.array_equal(a[key], b[key])
    for m in range(3):
        assert np.array_equal(a["u"][m], b["u"][m])
        assert np.array_equal(a["phi"][m], b["phi"][m])


def _accel(prm, rho, u, p, Ysum):
    h = prm.h
    visc = ops.div_stress(u, prm.mu, h)
    return [(visc[m] - ops.Gc(p, m, h)) / (rho * (1.0 + Ysum)) for m in range(3)]


@pytest.mark.parametrize("n_corr", [1, 2])
def test_momentum_exchange_identity(n_corr):
    """sum rho^{K-1} u^K - sum rho^n u^n = (dt/2) sum (f^n + f^{K-1}) exactly, K = n_corr.

    The corrected velocity is HbyA - (dt/rho^{K-1}) Gc p^K with HbyA = (rho^n u^n + dt R^K) /
    rho^{K-1} and R^K = (L^n + f^n + L^{K-1} + f^{K-1}) / 2: the divergence-form L and the periodic
    difference Gc sum to zero, the reaction forces do not.  f^n = -(rho^n Ysum) a^n; the first
    corrector's f^0 = -(rho^0 Ysum) a^n (rho^0 = rho^n - dt D phi^n), the second's
    f^1 = -(rho^1 Ysum) a^1 with the first corrector's rho^1, u^1, p^1.  Pins the sign, the 1/2,
    which density multiplies which acceleration, and the acceleration used after each corrector.
    """
    N = 8
    dt = 0.02
    prm = piso.Params(N=N, tau_p=[0.05, 0.1], Y0=[0.1, 0.1], n_corr=n_corr, p_tol=1e-12,
                      coupling=piso.TWO_WAY)
    st = loaded_state(prm, 7)
    Ysum = st["Y"][0] + st["Y"][1]
    a_n = _accel(prm, st["rho"], st["u"], st["p"], Ysum)
    if n_corr == 1:
        rho_prev = st["rho"] - dt * ops.D(st["phi"], prm.h)
        a_prev = a_n
    else:
        prm1 = piso.Params(N=N, tau_p=[0.05, 0.1], Y0=[0.1, 0.1], n_corr=1, p_tol=1e-12,
                           coupling=piso.TWO_WAY)
        s1, info1 = piso.step(prm1, st, dt=dt)
        rho_prev = s1["rho"]
        a_prev = _accel(prm, s1["rho"], s1["u"], info1["p_iter"], Ysum)
    new, _ = piso.step(prm, st, dt=dt)
    for m in range(3):
        got = np.sum(rho_prev * new["u"][m]) - np.sum(st["rho"] * st["u"][m])
        impulse = 0.5 * dt * np.sum(-(st["rho"] * Ysum) * a_n[m] - (rho_prev * Ysum) * a_prev[m])
        scale = np.sum(np.abs(st["rho"] * st["u"][m]))
        assert abs(impulse) > 1e-6 * scale  # seven orders above the tolerance below
        assert abs(got - impulse) <= 2e-13 * scale


def _acoustic_omega(N, dt, Y, coupling):
    eps = 1e-4
    x, y, z, h = grid(N)
    prm = piso.Params(N=N, nu=0.0, tau_p=[0.0], Y0=[Y], dt_max=dt, p_tol=1e-13, coupling=coupling)
    st = piso.make_state(prm, 1 + eps * np.cos(x), [0 * x] * 3, [np.full_like(x, Y)])
    for _ in range(int(round(1.0 / dt))):
        st, _info = piso.step(prm, st)
    a = np.sum((st["rho"] - 1) * np.cos(x)) / np.sum(np.cos(x) ** 2)
    return math.acos(a / eps) / st["t"]


def test_effective_sound_speed():
    """Uniform loading Y (Marble limit tau_p = 0, Y stays uniform): a k = 1 acoustic wave runs at
    c / sqrt(1 + Y).  The frequency ratio to the unloaded gas on the same grid and step tends to
    1 / sqrt(1 + Y) at first order in dt (the reaction force lags by one corrector); a wrong sign
    gives sqrt((1 + Y) / (1 + 3 Y)) - 1 = -15 %, the gas inertia alone in a gives +12 %."""
    Y = 0.25
    err = []
    for dt in (0.02, 0.01):
        w1 = _acoustic_omega(8, dt, Y, piso.ONE_WAY)
        w2 = _acoustic_omega(8, dt, Y, piso.TWO_WAY)
        err.append(w2 / w1 * math.sqrt(1 + Y) - 1)
    assert abs(err[1]) < 2e-4
    assert 1.6 < err[0] / err[1] < 2.4


def _shear_rate(dt, Y, coupling, N=8, nu=0.05, nsteps=20):
    x, y, z, h = grid(N)
    prm = piso.Params(N=N, nu=nu, tau_p=[0.0], Y0=[Y], dt_max=dt, p_tol=1e-13, coupling=coupling)
    st = piso.make_state(prm, np.ones_like(x), [1e-3 * np.sin(y), 0 * x, 0 * x], [np.full_like(x, Y)])
    ke0 = diag.diagnostics(st["rho"], st["u"], h)["ke_u"]
    for _ in range(nsteps):
        st, _ = piso.step(prm, st)
    ke = diag.diagnostics(st["rho"], st["u"], h)["ke_u"]
    return -math.log(ke / ke0) / st["t"]


def test_mixture_viscosity():
    """A shear wave u_x = A sin y under uniform loading Y decays at the mixture's kinematic
    viscosity nu / (1 + Y): the rate ratio to the unloaded gas tends to 1 / (1 + Y), here at
    second order in dt (the viscous operator of the reaction force is the momentum equation's)."""
    Y = 0.25
    err = []
    for dt in (0.04, 0.02):
        r1 = _shear_rate(dt, Y, piso.ONE_WAY)
        r2 = _shear_rate(dt, Y, piso.TWO_WAY)
        err.append(r2 / r1 * (1 + Y) - 1)
    assert abs(err[1]) < 2e-8
    assert 3.2 < err[0] / err[1] < 4.8


@pytest.mark.parametrize("closure,model", [(piso.FOURIER, piso.EQUILIBRIUM), (piso.BAROTROPIC, piso.TWO_FLUID)])
def test_two_way_scope(closure, model):
    """Two-way coupling is defined for the barotropic closure and the equilibrium dust model."""
    prm = piso.Params(N=8, closure=closure, dust_model=model, coupling=piso.TWO_WAY, tau_p=[0.05], Y0=[0.1])
    x, y, z, h = grid(8)
    one = np.ones_like(x)
    st = piso.make_state(prm, one, [0 * x] * 3, [0.1 * one], one if closure == piso.FOURIER else None,
                         V=[[0 * x] * 3] if model == piso.TWO_FLUID else None)
    with pytest.raises(ValueError):
        piso.step(prm, st, dt=0.01)
