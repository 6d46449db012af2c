"""Eulerian two-fluid dust phase (FP64): every dust class with a velocity of its own.

Test infrastructure (see ``oracle/__init__``).

Sec. 2 par. 2 of the paper sets its Equilibrium-Eulerian model (particle
velocity u_p = u - tau_p Du/Dt, a first-order expansion in the Stokes number)
against the full Eulerian two-phase model, in which the particle phase has
momentum of its own.  The paper prints no equations for either; the reading
adopted here is the dilute, pressureless, one-way coupled two-fluid model
(the gas is not loaded by the dust, as in the equilibrium reading), for each
class j with bulk density sigma = rho Y and velocity V:

    d sigma / dt + div(sigma V) = 0
    d (sigma V) / dt + div(sigma V V) = sigma (u - V) / tau_p     (Stokes drag)

Discretisation, after the gas step n -> n+1 (the gas does not depend on the
dust), with the operators of ``ops``:

* dust face flux of the carrier mass  phi_v,d = phi_d + I4_d(rho) I4_d(V_d - u_d)
  (the gas flux plus the interpolated slip; with V = u - tau_p a it is the
  equilibrium model's particle flux phi - tau_p I4(rho) I4(a));
  dust mass flux F_d = phi_v,d I4_d(Y); momentum flux G_dm = F_d I4_d(V_m);
* predictor: sigma* = sigma^n - dt D(F^n),  m* = sigma^n V^n - dt D(G^n),
  corrector: sigma^{n+1} = sigma^n - dt/2 [D(F^n) + D(F*)], m likewise, F*
  and G* from the gas at n+1 and the predicted dust (Heun, second order);
* drag implicit (backward Euler, L-stable): after each stage
      V = u^{n+1} + (m / sigma - u^{n+1}) tau_p / (tau_p + dt),
  so a uniform slip decays by tau_p / (tau_p + dt) per step and V -> u^{n+1}
  as tau_p -> 0;  Y = sigma / rho^{n+1}.

Parity pins (tests/test_oracle_twofluid.py): the uniform-slip relaxation
factor per step in closed form and its first-order convergence to
exp(-t/tau_p); exact conservation of dust mass and the exact momentum budget
(the change of sum sigma V equals the summed drag); the tracer limit
tau_p -> 0 (V = u, passive advection in a uniform stream converging to the
semi-discrete solution at second order); the first-order agreement with the
Equilibrium-Eulerian model as dt -> 0 (the response of Y to tau_p).
"""
import numpy as np

from . import ops


def dust_fluxes(phi, rho, u, Y, V, h):
    """D(F) and D(G_m) of one class at one level (cell fields)."""
    phv = [phi[d] + ops.I4(rho, d) * ops.I4(V[d] - u[d], d) for d in range(3)]
    F = [phv[d] * ops.I4(Y, d) for d in range(3)]
    DF = ops.D(F, h)
    DG = [ops.D([F[d] * ops.I4(V[m], d) for d in range(3)], h) for m in range(3)]
    return DF, DG


def drag(sig, mom, u, dt, tau):
    """Backward-Euler Stokes drag toward u: V = u + (mom/sig - u) tau / (tau + dt)."""
    r = tau / (tau + dt)
    return [u[m] + (mom[m] / sig - u[m]) * r for m in range(3)]


def step_class(gas_n, gas_1, Y_n, V_n, tau, dt, h):
    """One step of one dust class.  gas_* = (rho, u, phi) at levels n and n+1.
    Returns (Y^{n+1}, V^{n+1})."""
    rho_n, u_n, phi_n = gas_n
    rho_1, u_1, phi_1 = gas_1
    sig_n = rho_n * Y_n
    mom_n = [sig_n * V_n[m] for m in range(3)]
    DFn, DGn = dust_fluxes(phi_n, rho_n, u_n, Y_n, V_n, h)
    sig_s = sig_n - dt * DFn
    mom_s = [mom_n[m] - dt * DGn[m] for m in range(3)]
    V_s = drag(sig_s, mom_s, u_1, dt, tau)
    Y_s = sig_s / rho_1
    DFs, DGs = dust_fluxes(phi_1, rho_1, u_1, Y_s, V_s, h)
    sig = sig_n - 0.5 * dt * (DFn + DFs)
    mom = [mom_n[m] - 0.5 * dt * (DGn[m] + DGs[m]) for m in range(3)]
    V = drag(sig, mom, u_1, dt, tau)
    return sig / rho_1, V
