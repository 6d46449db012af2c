"""Pins for the oracle's Eulerian two-fluid dust phase (oracle/twofluid.py).

Sec. 2 par. 2 of the paper contrasts the Equilibrium-Eulerian model with the
full Eulerian two-phase model, where the particles carry momentum of their
own; the discrete reading is stated in oracle/twofluid.py.  Pins:

* uniform slip relaxation: a uniform gas (which stays uniform) and a uniform
  dust slip s: after n steps the slip is s (tau / (tau + dt))^n exactly, and
  it converges to s exp(-t / tau) at first order in dt;
* exact conservation of every class's dust mass, and the exact momentum
  budget sum sigma V (n+1) - sum sigma V (n) = (dt / tau) sum sigma (u - V)
  at n+1 (the flux divergences sum to zero);
* tracer limit tau -> 0: V = u, and Y = 0.01 + a sin x in a uniform stream is
  carried at the speed of the fourth-order flux symbol, converging to that
  semi-discrete solution at second order in dt;
* first-order agreement with the Equilibrium-Eulerian model: from the same
  state (dust started at u - tau Du/Dt, uniform Y) the response of Y to a
  small tau matches the equilibrium model's response up to a difference that
  halves with dt (0.5 % at dt = 0.01).
"""
import math

import numpy as np
import pytest

from oracle import piso, twofluid

from .test_oracle_piso import grid, random_state


def two_fluid_state(prm, seed):
    """A random state with the dust started at u - tau Du/Dt (the equilibrium particle velocity)."""
    st = random_state(prm, seed)
    a = piso.accel(prm, st["rho"], st["u"], st["p"])
    st["V"] = [[st["u"][m] - tau * a[m] for m in range(3)] for tau in prm.tau_p]
    return st


def test_uniform_slip_relaxation_closed_form():
    N, tau = 8, 0.05
    ones = np.ones((N, N, N))
    U, s = (0.2, -0.1, 0.05), (0.03, 0.01, -0.02)
    for dt, nsteps in ((0.02, 10), (0.01, 20), (0.005, 40)):
        prm = piso.Params(N=N, tau_p=[tau], Y0=[0.01], dust_model=piso.TWO_FLUID, dt_max=dt)
        u = [c * ones for c in U]
        st = piso.make_state(prm, 1.3 * ones, u, [0.01 * ones], V=[[(U[m] + s[m]) * ones for m in range(3)]])
        for _ in range(nsteps):
            st, _ = piso.step(prm, st, dt=dt)
        r = (tau / (tau + dt)) ** nsteps
        for m in range(3):
            np.testing.assert_allclose(st["u"][m], U[m] * ones, rtol=0, atol=1e-14)
            np.testing.assert_allclose(st["V"][0][m] - U[m], s[m] * r * ones, rtol=1e-12, atol=1e-16)
    # first order in dt toward exp(-t / tau), t = 0.2
    errs = []
    for dt in (0.02, 0.01, 0.005):
        n = int(round(0.2 / dt))
        errs.append(abs((tau / (tau + dt)) ** n - math.exp(-0.2 / tau)))
    assert 1.8 < errs[0] / errs[1] < 2.4 and 1.8 < errs[1] / errs[2] < 2.4


def test_dust_mass_conservation_and_momentum_budget():
    prm = piso.Params(N=12, tau_p=[0.02, 0.1, 0.3], Y0=[0.02] * 3, dust_model=piso.TWO_FLUID, p_tol=1e-12)
    st = two_fluid_state(prm, 5)
    for _ in range(2):
        t0 = piso.totals(prm, st)
        new, info = piso.step(prm, st)
        t1 = piso.totals(prm, new)
        vol = prm.h ** 3
        for j, tau in enumerate(prm.tau_p):
            assert abs(t1["dust"][j] - t0["dust"][j]) <= 1e-14 * t0["dust"][j]
            sig = new["rho"] * new["Y"][j]
            for m in range(3):
                drag = vol * info["dt"] / tau * float(np.sum(sig * (new["u"][m] - new["V"][j][m])))
                change = t1["dust_momentum"][j][m] - t0["dust_momentum"][j][m]
                scale = vol * float(np.sum(np.abs(sig * new["V"][j][m])))
                assert abs(change - drag) <= 1e-13 * scale, (j, m, change, drag)
        st = new


def _advected_two_fluid_error(N, dt, U=0.5, amp=1e-3):
    x, y, z, h = grid(N)
    prm = piso.Params(N=N, nu=0.0, tau_p=[1e-14], Y0=[0.0], dt_max=dt, dust_model=piso.TWO_FLUID)
    st = piso.make_state(prm, np.ones_like(x), [U + 0 * x, 0 * x, 0 * x], [0.01 + amp * np.sin(x)])
    for _ in range(int(round(1.0 / dt))):
        st, _info = piso.step(prm, st, dt=dt)
    for m in range(3):
        assert np.max(np.abs(st["V"][0][m] - st["u"][m])) < 1e-14
    Y = st["Y"][0] - 0.01
    a = np.sum(Y * np.sin(x)) / np.sum(np.sin(x) ** 2) / amp
    b = np.sum(Y * np.cos(x)) / np.sum(np.cos(x) ** 2) / amp
    # semi-discrete exact solution: sin(x - U k* t), k* the symbol of D o I4 at k = 1
    ks = (2 * np.sin(h / 2) / h) * (9 * np.cos(h / 2) - np.cos(3 * h / 2)) / 8
    th = U * ks * st["t"]
    return float(np.hypot(a - np.cos(th), b + np.sin(th)))


def test_tracer_limit_advects_at_second_order():
    e1, e2 = _advected_two_fluid_error(16, 0.1), _advected_two_fluid_error(16, 0.05)
    assert e1 < 5e-4
    assert 3.5 < e1 / e2 < 4.5


def _response(model, tau, dt, seed=11):
    prm = piso.Params(N=12, tau_p=[tau], Y0=[0.0], p_tol=1e-13, dust_model=model)
    st = random_state(prm, seed)
    # uniform Y: the dust phase's momentum convection then has the gas's discrete form, so the two
    # models differ only in how time is discretised (a grid-scale Y adds a spatial difference)
    st["Y"] = [np.full_like(st["rho"], 0.01)]
    if model == piso.TWO_FLUID:  # V = u - tau Du/Dt, the equilibrium model's particle velocity
        a = piso.accel(prm, st["rho"], st["u"], st["p"])
        st["V"] = [[st["u"][m] - tau * a[m] for m in range(3)]]
    new, _ = piso.step(prm, st, dt=dt)
    return new["Y"][0]


def test_first_order_agreement_with_the_equilibrium_model():
    """(Y(tau) - Y(0)) / tau of both models; their relative difference falls in
    proportion to dt (the two-fluid slip carries a kinematic Du/Dt over the step,
    the equilibrium model the dynamic one at the iterate: both first order)."""
    tau = 1e-5
    diffs = []
    for dt in (0.01, 0.005, 0.0025):
        eq = (_response(piso.EQUILIBRIUM, tau, dt) - _response(piso.EQUILIBRIUM, 0.0, dt)) / tau
        tf = (_response(piso.TWO_FLUID, tau, dt) - _response(piso.TWO_FLUID, 1e-14, dt)) / tau
        diffs.append(float(np.linalg.norm(tf - eq) / np.linalg.norm(eq)))
    assert diffs[0] < 1e-2
    assert 1.9 < diffs[0] / diffs[1] < 2.1 and 1.9 < diffs[1] / diffs[2] < 2.1, diffs


def test_drag_limits():
    """The backward-Euler drag: V -> u as tau -> 0 and V -> m / sigma as tau -> inf."""
    rng = np.random.default_rng(3)
    sig = 1.0 + 0.1 * rng.random((4, 4, 4))
    mom = [rng.standard_normal((4, 4, 4)) for _ in range(3)]
    u = [rng.standard_normal((4, 4, 4)) for _ in range(3)]
    v0 = twofluid.drag(sig, mom, u, 0.1, 1e-300)
    vi = twofluid.drag(sig, mom, u, 0.1, 1e300)
    for m in range(3):
        np.testing.assert_allclose(v0[m], u[m], rtol=1e-15)
        np.testing.assert_allclose(vi[m], mom[m] / sig, rtol=0, atol=1e-15 * np.max(np.abs(u[m])))
