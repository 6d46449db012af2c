"""One compressible PISO step of Equilibrium-Eulerian dusty decaying HIT (FP64).

Test infrastructure (see ``oracle/__init__``).  A nonlinear step has no
closed form, so this function is the definition of the discrete step; every
term of it is pinned by at least one of the tests listed at the end of this
header.

Paper passages it restates (arXiv:1404.0959):

* Sec. 2, par. 1: pressure-based PISO solver with fourth-order central
  interpolation and an adaptive time step.
* Sec. 2, par. 2, footnotes: barotropic closure p ~ rho^gamma (no energy
  equation) or Fourier closure (energy equation with q = -k grad T).
* Sec. 2, par. 2: Equilibrium-Eulerian particle velocity, first order in the
  Stokes number with Stokes drag: u_p = u - tau_p Du/Dt ("kinematic
  quasi-equilibrium").
* Sec. 2, par. 3 and footnote: tau_p = 0 is Marble's dusty gas (u_p = u).
* Two-way coupling (the dusty-gas mixture of the Sec. 2 par. 3 footnote's
  reference): the dust drag acts back on the gas.  With the first-order
  particle velocity the drag per unit dust mass is the gas acceleration a, so
  the gas momentum gains f = -rho Ysum a (Ysum = sum_j Y_j), and a itself
  solves rho a = D tau - Gc p + f, i.e. a = (D tau - Gc p) / (rho (1 + Ysum)):
  the mixture inertia of Marble's dusty gas.

The paper gives no equations; the discrete algorithm below ("Algorithm O") is
this project's reading, in the order it is computed.  Symbols: operators from
``oracle.ops``; n = old level; k = corrector iterate; psi = rho/(gamma p)
frozen at level n; mu = nu (reference density 1).

 a1  dt = min(CFL h / max_i sum_d |u_d|, growth * dt_prev, dt_max)
 a3  rho0 = rho^n - dt D(phi^n)
     R^n  = L(u^n, phi^n)                    [+ f^n = -(rho^n Ysum) a^n  two-way]
     u*   = (rho^n u^n + dt (R^n - Gc p^n)) / rho0
     n-level dust and energy flux divergences (a7, a8)
     iterates: (u, phi, p, rho, Y, E)^0 = (u*, phi^n, p^n, rho0, Y^n, E^n)
 for k = 1 .. n_corr:
 a4  R^k   = (R^n + L(u^{k-1}, phi^{k-1}) [- (rho^{k-1} Ysum) A]) / 2
                (two-way: A = a^n in the first corrector, a^{k-1} after)
     HbyA  = (rho^n u^n + dt R^k) / rho^{k-1}
     phiH  = I4(rho^{k-1}) I4(HbyA)          (per face direction)
     phi*  = phiH - dt G2(p^{k-1})
     b     = -[(rho^{k-1} - rho^n)/dt + D(phi^n)/2 + D(phi*)/2]
 a5  M p' = b,  M p' = psi p'/dt - (dt/2) D(G2 p')
                [+ (1/2) D(I4(psi p') I4(HbyA))  when transonic]
     (Jacobi-PCG; BiCGStab when transonic; flexible CG with a given
      preconditioner; flexible GMRES(20) for either operator when fgmres)
 a6  p^k   = p^{k-1} + p'
     phi^k = phi* - dt G2(p')  [+ I4(psi p') I4(HbyA) when transonic]
     u^k   = HbyA - (dt / rho^{k-1}) Gc(p^k)
     rho^k = rho^n - (dt/2) [D(phi^n) + D(phi^k)]
 a7  a^k     = (-Gc p^k + D tau(u^k)) / rho^k                (Du/Dt)
              [/ (rho^k (1 + Ysum)) two-way; Ysum = sum_j Y_j^n over the step]
     phi_p^k = phi^k - tau_p I4(rho^k) I4(a^k)             (per class)
     (rho Y)^k = rho^n Y^n - (dt/2) [D(phi_p^n I4(Y^n)) + D(phi_p^k I4(Y^{k-1}))]
 a8  Fourier: F_E = phi I4(E + p/rho) - sum_m tau_dm I4(u_m) - kappa G4(T)
     (rho E)^k = rho^n E^n - (dt/2) [D(F_E^n) + D(F_E^k)]
     level k uses E^{k-1}, p^k/rho^k and T = p^k / (rho^k R)
 end
     closure: barotropic p = rho^gamma / gamma;
              Fourier T = (E - |u|^2/2) / c_v, p = rho R T.

Constants (Fourier): R = 1/gamma, c_v = R/(gamma-1), c_p = gamma c_v,
kappa = mu c_p / Pr, so the reference state rho = T = 1 has p = 1/gamma and
sound speed 1 in both closures.

Pins (tests/test_oracle_piso.py): Taylor-Green viscous decay rate against the
discrete and the analytic rate; exact conservation of mass, dust mass and
total energy; uniform state stays uniform; tau_p = 0 passive tracer; first
order response in tau_p; closed-form initial dust drift for a pressure and
for a dilatational velocity perturbation; isobaric heat-conduction decay;
viscous heating of a shear wave where it dissipates (Fourier); passive dust
advection at second order in time;
acoustic wave speed c = 1; psi c^2 = 1 with c^2 the isentropic derivative of
the closure's EOS; the adaptive step's Courant number, growth limit and cap;
with one corrector, sum rho^0 u^{n+1} = sum rho^n u^n exactly.
Two-way coupling (tests/test_oracle_twoway.py): Ysum = 0 gives the one-way
step bit for bit; the momentum the gas gains in the last corrector equals
dt/2 sum (f^n + f^{K-1}) exactly; the acoustic period grows by sqrt(1 + Y)
and the shear-wave decay rate falls by 1 + Y (Marble's effective gas) as
dt -> 0.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import ops, twofluid
from .krylov import bicgstab, fcg, fgmres, pcg

BAROTROPIC = 0
FOURIER = 1
EQUILIBRIUM = 0  # dust model: particle velocity u - tau_p Du/Dt (Sec. 2 par. 2)
TWO_FLUID = 1    # dust model: every class with its own momentum (oracle/twofluid.py)
ONE_WAY = 0      # coupling: the dust does not act on the gas
TWO_WAY = 1      # coupling: the drag's reaction -rho Ysum a on the gas (equilibrium dust, barotropic)


@dataclass
class Params:
    N: int = 32
    closure: int = BAROTROPIC
    gamma: float = 1.4
    Pr: float = 0.7
    nu: float = 0.005
    tau_p: list = field(default_factory=lambda: [0.05])
    Y0: list = field(default_factory=lambda: [0.01])
    mach_rms: float = 0.2
    k0: float = 4.0
    seed: int = 0
    cfl: float = 0.5
    dt_growth_max: float = 1.2
    dt_max: float = math.inf
    n_corr: int = 2
    p_tol: float = 1e-10
    p_maxit: int = 500
    transonic: bool = False
    fgmres: bool = False  # flexible GMRES(20) for every solve (any operator)
    dust_model: int = EQUILIBRIUM
    coupling: int = ONE_WAY

    @property
    def h(self):
        return 2.0 * math.pi / self.N

    @property
    def mu(self):
        return self.nu

    @property
    def R(self):
        return 1.0 / self.gamma

    @property
    def cv(self):
        return self.R / (self.gamma - 1.0)

    @property
    def cp(self):
        return self.gamma * self.cv

    @property
    def kappa(self):
        return self.mu * self.cp / self.Pr

    @property
    def n_dust(self):
        return len(self.tau_p)


def eos_pressure(prm, rho, T=None):
    """Barotropic p = rho^gamma/gamma, or Fourier p = rho R T."""
    if prm.closure == BAROTROPIC:
        return rho ** prm.gamma / prm.gamma
    return rho * prm.R * T


def compressibility(prm, rho, p):
    """psi = rho/(gamma p) = 1/c^2, the isentropic compressibility (both closures)."""
    return rho / (prm.gamma * p)


def face_flux(rho, u):
    """Initial mass flux phi_d = I4(rho) I4(u_d)."""
    return [ops.I4(rho, d) * ops.I4(u[d], d) for d in range(3)]


def make_state(prm, rho, u, Y, T=None, phi=None, V=None):
    """Assemble a state dict; p from the closure, phi = I4(rho) I4(u) unless given.
    Two-fluid dust: V[j] = the velocity of class j (the gas velocity unless given)."""
    rho = np.asarray(rho, dtype=np.float64)
    u = [np.asarray(c, dtype=np.float64) for c in u]
    Y = [np.asarray(y, dtype=np.float64) for y in Y]
    if prm.closure == FOURIER:
        T = np.asarray(T, dtype=np.float64)
    p = eos_pressure(prm, rho, T)
    if phi is None:
        phi = face_flux(rho, u)
    st = {"rho": rho, "u": u, "phi": phi, "p": p, "Y": Y, "T": T,
          "t": 0.0, "dt_prev": math.inf}
    if prm.dust_model == TWO_FLUID:
        st["V"] = [[np.array(c, dtype=np.float64) for c in (V[j] if V is not None else u)] for j in range(len(Y))]
    return st


def initial_state(prm):
    """Spectral HIT initial condition: rho = 1, T = 1, uniform Y, random u."""
    from .ic import spectral_velocity
    N = prm.N
    u = spectral_velocity(N, prm.k0, prm.mach_rms, prm.seed)
    rho = np.ones((N, N, N))
    Y = [np.full((N, N, N), float(y)) for y in prm.Y0]
    T = np.ones((N, N, N)) if prm.closure == FOURIER else None
    return make_state(prm, rho, u, Y, T)


def time_step(prm, u, dt_prev):
    """a1: CFL-limited step with growth limit."""
    umax = float(np.max(np.abs(u[0]) + np.abs(u[1]) + np.abs(u[2])))
    dt = prm.cfl * prm.h / umax if umax > 0.0 else math.inf
    return min(dt, prm.dt_growth_max * dt_prev, prm.dt_max)


def accel(prm, rho, u, p, Ysum=None):
    """Du/Dt in dynamic form: (-Gc p + D tau(u)) / rho, three components;
    with the dust's reaction (two-way coupling) the inertia is rho (1 + Ysum)."""
    h = prm.h
    visc = ops.div_stress(u, prm.mu, h)
    inertia = rho if Ysum is None else rho * (1.0 + Ysum)
    return [(-ops.Gc(p, m, h) + visc[m]) / inertia for m in range(3)]


def reaction(rho, Ysum, a):
    """Two-way coupling: the force of the dust drag on the gas, f = -(rho Ysum) a."""
    return [-(rho * Ysum) * a[m] for m in range(3)]


def dust_sum(Y):
    """Ysum = sum_j Y_j, summed in class order."""
    s = Y[0]
    for j in range(1, len(Y)):
        s = s + Y[j]
    return s


def particle_flux(prm, phi, rho, a, j):
    """Equilibrium-Eulerian particle mass flux phi_p = phi - tau_p I4(rho) I4(a)."""
    tp = prm.tau_p[j]
    return [phi[d] - tp * ops.I4(rho, d) * ops.I4(a[d], d) for d in range(3)]


def energy_flux(prm, phi, u, rho, p, E, T):
    """Total-energy face flux phi I4(E + p/rho) - sum_m tau_dm I4(u_m) - kappa G4(T)."""
    h = prm.h
    tau = ops.stress(u, prm.mu, h)
    H = E + p / rho
    F = []
    for d in range(3):
        work = tau[d][0] * ops.I4(u[0], d) + tau[d][1] * ops.I4(u[1], d) + tau[d][2] * ops.I4(u[2], d)
        F.append(phi[d] * ops.I4(H, d) - work - prm.kappa * ops.G4(T, d, h))
    return F


def helmholtz(prm, psi, dt, HbyA=None):
    """Return (matvec, jacobi_diag) of the pressure-correction operator M."""
    h = prm.h

    def matvec(x):
        lap = ops.D([ops.G2(x, d, h) for d in range(3)], h)
        y = psi * x / dt - 0.5 * dt * lap
        if HbyA is not None:
            px = psi * x
            y = y + 0.5 * ops.D([ops.I4(px, d) * ops.I4(HbyA[d], d) for d in range(3)], h)
        return y

    diag = psi / dt + 3.0 * dt / (h * h)
    return matvec, diag


def solve(prm, matvec, b, diag, precond=None):
    if prm.fgmres:
        pre = None if precond is None else (lambda v, it: precond(v))
        return fgmres(matvec, b, pre, diag, prm.p_tol, prm.p_maxit, m=20)
    if precond is not None:
        return fcg(matvec, b, precond, diag, prm.p_tol, prm.p_maxit)
    if prm.transonic:
        return bicgstab(matvec, b, diag, prm.p_tol, prm.p_maxit)
    return pcg(matvec, b, diag, prm.p_tol, prm.p_maxit)


def step(prm, state, precond=None, dt=None):
    """Advance ``state`` by one PISO step; returns (new_state, info).

    ``precond`` (optional) is a callable r -> z used inside flexible CG.
    ``dt`` (optional) overrides the adaptive step (tests only).
    """
    h = prm.h
    nd = prm.n_dust
    rho_n, u_n, phi_n, p_n = state["rho"], state["u"], state["phi"], state["p"]
    Y_n, T_n = state["Y"], state["T"]
    fourier = prm.closure == FOURIER

    # a1: adaptive time step, psi frozen at level n
    if dt is None:
        dt = time_step(prm, u_n, state["dt_prev"])
    psi = compressibility(prm, rho_n, p_n)

    eq_dust = prm.dust_model == EQUILIBRIUM
    two_way = prm.coupling == TWO_WAY and nd > 0
    if two_way and (fourier or not eq_dust):
        raise ValueError("two-way coupling: barotropic closure and equilibrium dust only")
    Ysum = dust_sum(Y_n) if two_way else None

    # a3: predictor
    divphi_n = ops.D(phi_n, h)
    rho0 = rho_n - dt * divphi_n
    a_n = accel(prm, rho_n, u_n, p_n, Ysum)
    R_n = ops.L(u_n, phi_n, prm.mu, h)
    if two_way:
        f_n = reaction(rho_n, Ysum, a_n)
        R_n = [R_n[m] + f_n[m] for m in range(3)]
    mom_n = [rho_n * u_n[m] for m in range(3)]
    u_star = [(mom_n[m] + dt * (R_n[m] - ops.Gc(p_n, m, h))) / rho0 for m in range(3)]

    FY_n = []
    for j in range(nd if eq_dust else 0):
        fp = particle_flux(prm, phi_n, rho_n, a_n, j)
        FY_n.append(ops.D([fp[d] * ops.I4(Y_n[j], d) for d in range(3)], h))
    if fourier:
        E_n = prm.cv * T_n + 0.5 * (u_n[0] ** 2 + u_n[1] ** 2 + u_n[2] ** 2)
        FE_n = ops.D(energy_flux(prm, phi_n, u_n, rho_n, p_n, E_n, T_n), h)

    rho_k, u_k, phi_k, p_k = rho0, u_star, phi_n, p_n
    Y_k = list(Y_n)
    E_k = E_n if fourier else None
    A = a_n  # the latest Du/Dt (two-way: the reaction force of the next assembly)
    iters = []
    res = []

    for _k in range(prm.n_corr):
        # a4: corrector assembly
        Lk = ops.L(u_k, phi_k, prm.mu, h)
        if two_way:
            f_k = reaction(rho_k, Ysum, A)
            Lk = [Lk[m] + f_k[m] for m in range(3)]
        R_k = [0.5 * (R_n[m] + Lk[m]) for m in range(3)]
        HbyA = [(mom_n[m] + dt * R_k[m]) / rho_k for m in range(3)]
        phiH = [ops.I4(rho_k, d) * ops.I4(HbyA[d], d) for d in range(3)]
        phistar = [phiH[d] - dt * ops.G2(p_k, d, h) for d in range(3)]
        b = -((rho_k - rho_n) / dt + 0.5 * divphi_n + 0.5 * ops.D(phistar, h))

        # a5: pressure-correction solve
        matvec, diag = helmholtz(prm, psi, dt, HbyA if prm.transonic else None)
        pc, it, rel_rec, rel_true = solve(prm, matvec, b, diag, precond)
        iters.append(it)
        res.append(rel_true)

        # a6: flux, velocity and density correction
        p_new = p_k + pc
        phi_new = []
        for d in range(3):
            f = phistar[d] - dt * ops.G2(pc, d, h)
            if prm.transonic:
                f = f + ops.I4(psi * pc, d) * ops.I4(HbyA[d], d)
            phi_new.append(f)
        u_new = [HbyA[m] - (dt / rho_k) * ops.Gc(p_new, m, h) for m in range(3)]
        rho_new = rho_n - 0.5 * dt * (divphi_n + ops.D(phi_new, h))

        # a7: particle velocity and dust transport
        a_k = accel(prm, rho_new, u_new, p_new, Ysum)
        A = a_k
        Y_new = [] if eq_dust else list(Y_k)
        for j in range(nd if eq_dust else 0):
            fp = particle_flux(prm, phi_new, rho_new, a_k, j)
            FY_k = ops.D([fp[d] * ops.I4(Y_k[j], d) for d in range(3)], h)
            rhoY = rho_n * Y_n[j] - 0.5 * dt * (FY_n[j] + FY_k)
            Y_new.append(rhoY / rho_new)

        # a8: energy (Fourier)
        if fourier:
            T_it = p_new / (rho_new * prm.R)
            FE_k = ops.D(energy_flux(prm, phi_new, u_new, rho_new, p_new, E_k, T_it), h)
            rhoE = rho_n * E_n - 0.5 * dt * (FE_n + FE_k)
            E_k = rhoE / rho_new

        rho_k, u_k, phi_k, p_k, Y_k = rho_new, u_new, phi_new, p_new, Y_new

    # closure
    if fourier:
        T_new = (E_k - 0.5 * (u_k[0] ** 2 + u_k[1] ** 2 + u_k[2] ** 2)) / prm.cv
        p_final = rho_k * prm.R * T_new
    else:
        T_new = None
        p_final = eos_pressure(prm, rho_k)

    new = {"rho": rho_k, "u": u_k, "phi": phi_k, "p": p_final, "Y": Y_k, "T": T_new,
           "t": state["t"] + dt, "dt_prev": dt}
    if not eq_dust:  # two-fluid dust after the gas step (the gas does not depend on it)
        new["Y"], new["V"] = [], []
        for j in range(nd):
            Yj, Vj = twofluid.step_class((rho_n, u_n, phi_n), (rho_k, u_k, phi_k), Y_n[j], state["V"][j],
                                         prm.tau_p[j], dt, h)
            new["Y"].append(Yj)
            new["V"].append(Vj)
    info = {"dt": dt, "iters": iters, "rel_res": res, "psi": psi, "p_iter": p_k}
    return new, info


def totals(prm, state):
    """Conserved totals (cell sums times h^3): mass, dust masses, total energy."""
    vol = prm.h ** 3
    rho = state["rho"]
    u = state["u"]
    out = {"mass": vol * float(np.sum(rho)),
           "dust": [vol * float(np.sum(rho * y)) for y in state["Y"]]}
    ke = 0.5 * rho * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    if prm.closure == FOURIER:
        out["energy"] = vol * float(np.sum(rho * prm.cv * state["T"] + ke))
    else:
        out["energy"] = vol * float(np.sum(ke))
    if state.get("V") is not None:
        out["dust_momentum"] = [[vol * float(np.sum(rho * y * v[m])) for m in range(3)]
                                for y, v in zip(state["Y"], state["V"])]
    return out
