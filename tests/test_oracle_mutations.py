"""The oracle's pins are sensitive: plausible mistakes planted in the oracle
(on the CPU, through monkeypatching) make at least one pin fail.

Each case names the mistake and the pin expected to catch it.
"""
import numpy as np
import pytest

from oracle import krylov, ops, piso

from . import test_oracle_ops as t_ops
from . import test_oracle_piso as t_piso
from . import test_oracle_solve as t_solve
from . import test_oracle_twoway as t_tw


def _bad_I4(f, d):
    return (-ops.at(f, d, -1) + 9.0 * f + 9.0 * ops.at(f, d, 1) - ops.at(f, d, 2)) / 15.9


def _bad_G4(f, d, h):
    return (ops.at(f, d, -1) - 27.0 * f + 27.0 * ops.at(f, d, 1) - ops.at(f, d, 2)) / (26.0 * h)


def _stress_no_dilatation(u, mu, h):
    tau = [[None] * 3 for _ in range(3)]
    for d in range(3):
        for m in range(3):
            tau[d][m] = mu * (ops.G4(u[m], d, h) + ops.I4(ops.Gc(u[d], m, h), d))
    return tau


def _stress_transposed(u, mu, h):
    div = ops.Gc(u[0], 0, h) + ops.Gc(u[1], 1, h) + ops.Gc(u[2], 2, h)
    tau = [[None] * 3 for _ in range(3)]
    for d in range(3):
        for m in range(3):
            t = ops.G4(u[m], d, h) + ops.I4(ops.Gc(u[m], d, h), d)
            if d == m:
                t = t - (2.0 / 3.0) * ops.I4(div, d)
            tau[d][m] = mu * t
    return tau


def _L_wrong_sign(u, phi, mu, h):
    visc = ops.div_stress(u, mu, h)
    return [ops.D([phi[d] * ops.I4(u[m], d) for d in range(3)], h) + visc[m] for m in range(3)]


def _eos_no_gamma_division(prm, rho, T=None):
    if prm.closure == piso.BAROTROPIC:
        return rho ** prm.gamma
    return rho * prm.R * T


def _accel_wrong_sign(prm, rho, u, p, Ysum=None):
    visc = ops.div_stress(u, prm.mu, prm.h)
    inertia = rho if Ysum is None else rho * (1.0 + Ysum)
    return [(ops.Gc(p, m, prm.h) + visc[m]) / inertia for m in range(3)]


def _accel_one_way_inertia(prm, rho, u, p, Ysum=None):
    visc = ops.div_stress(u, prm.mu, prm.h)
    return [(-ops.Gc(p, m, prm.h) + visc[m]) / rho for m in range(3)]


def _reaction_wrong_sign(rho, Ysum, a):
    return [(rho * Ysum) * a[m] for m in range(3)]


def _energy_no_pressure_work(prm, phi, u, rho, p, E, T):
    tau = ops.stress(u, prm.mu, prm.h)
    F = []
    for d in range(3):
        work = sum(tau[d][m] * ops.I4(u[m], d) for m in range(3))
        F.append(phi[d] * ops.I4(E, d) - work - prm.kappa * ops.G4(T, d, prm.h))
    return F


def _L_advective(u, phi, mu, h):
    # convection as (face flux averaged to the cell) . Gc(u): not a divergence
    visc = ops.div_stress(u, mu, h)
    out = []
    for m in range(3):
        adv = sum(0.5 * (phi[d] + ops.at(phi[d], d, -1)) * ops.Gc(u[m], d, h) for d in range(3))
        out.append(-adv + visc[m])
    return out


def _energy_no_viscous_work(prm, phi, u, rho, p, E, T):
    H = E + p / rho
    return [phi[d] * ops.I4(H, d) - prm.kappa * ops.G4(T, d, prm.h) for d in range(3)]


def _givens_transposed(a, b):
    if b == 0.0:
        return 1.0, 0.0
    h = float(np.hypot(a, b))
    return b / h, a / h


def _dt_euclidean(prm, u, dt_prev):
    umax = float(np.max(np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)))
    return min(prm.cfl * prm.h / umax, prm.dt_growth_max * dt_prev, prm.dt_max)


def _psi_isothermal(prm, rho, p):
    return rho / p


def _neumann1_without_the_two(matvec, diag):
    return lambda v: (v - matvec(v / diag)) / diag


def _neumann1_left_right_swapped(matvec, diag):
    return lambda v: 2.0 * v / diag - matvec(v) / diag ** 2


CASES = [
    ("I4 normalisation", ops, "I4", _bad_I4, lambda: t_ops.test_symbols(16, 1, 0)),
    ("G4 normalisation", ops, "G4", _bad_G4, lambda: t_ops.test_order_G4()),
    ("stress without 2/3 div", ops, "stress", _stress_no_dilatation,
     lambda: t_ops.test_viscous_stress_closed_form()),
    ("stress transposed gradient", ops, "stress", _stress_transposed,
     lambda: t_ops.test_viscous_stress_closed_form()),
    ("convection sign", ops, "L", _L_wrong_sign, lambda: t_ops.test_convection_closed_form()),
    ("advective convection", ops, "L", _L_advective,
     lambda: t_piso.test_single_corrector_momentum_identity(piso.BAROTROPIC, 0)),
    ("barotropic EOS without 1/gamma", piso, "eos_pressure", _eos_no_gamma_division,
     lambda: t_piso.test_acoustic_wave_speed()),
    ("Euclidean Courant number", piso, "time_step", _dt_euclidean,
     lambda: t_piso.test_adaptive_time_step_courant_number_and_growth()),
    ("Givens rotation with swapped entries", krylov, "_givens", _givens_transposed,
     lambda: t_solve.test_fgmres_minimises_residual_over_its_directions(3)),
    ("Neumann polynomial without the factor 2", krylov, "neumann1", _neumann1_without_the_two,
     lambda: t_solve.test_neumann1_is_two_jacobi_sweeps()),
    ("Neumann polynomial with M D^-1 D^-1 order", krylov, "neumann1", _neumann1_left_right_swapped,
     lambda: t_solve.test_neumann1_symmetric_positive_with_squared_jacobi_spectrum(0.4)),
    ("isothermal compressibility", piso, "compressibility", _psi_isothermal,
     lambda: t_piso.test_psi_is_inverse_isentropic_sound_speed_squared(piso.FOURIER)),
    ("Du/Dt pressure sign", piso, "accel", _accel_wrong_sign,
     lambda: t_piso.test_dust_drift_pressure_closed_form()),
    ("energy flux without viscous work", piso, "energy_flux", _energy_no_viscous_work,
     lambda: t_piso.test_viscous_heating_pattern()),
    ("enthalpy flux without p/rho", piso, "energy_flux", _energy_no_pressure_work,
     lambda: t_piso.test_isobaric_heat_conduction_rate()),
    ("two-way Du/Dt with the gas inertia only", piso, "accel", _accel_one_way_inertia,
     lambda: t_tw.test_mixture_viscosity()),
    ("two-way reaction force with the wrong sign", piso, "reaction", _reaction_wrong_sign,
     lambda: t_tw.test_effective_sound_speed()),
    ("two-way reaction force with the wrong sign (momentum)", piso, "reaction", _reaction_wrong_sign,
     lambda: t_tw.test_momentum_exchange_identity(1)),
]


@pytest.mark.parametrize("name,mod,attr,bad,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, mod, attr, bad, pin):
    monkeypatch.setattr(mod, attr, bad)
    with pytest.raises(AssertionError):
        pin()


def test_dropped_trapezoid_average_is_caught(monkeypatch):
    """R^k = L(u^{k-1}) instead of (R^n + L)/2: first order in time, TG rate moves."""
    orig_L = ops.L
    calls = {"n": 0}

    def L_counting(u, phi, mu, h):
        calls["n"] += 1
        out = orig_L(u, phi, mu, h)
        # the predictor call (first of each step) is kept; corrector calls return 2L - R^n
        # which turns (R^n + L)/2 into L
        return out

    monkeypatch.setattr(ops, "L", L_counting)
    r, nu, h = t_piso._tg_rate(16, nsteps=4)
    assert abs(r / (6 * nu * t_piso.s1(h)) - 1) < 2e-5  # unmodified: passes

    state = {}

    def L_biased(u, phi, mu, h):
        out = orig_L(u, phi, mu, h)
        if "Rn" not in state or state.get("fresh", False):
            state["Rn"] = out
            state["fresh"] = False
            return out
        return [2 * out[m] - state["Rn"][m] for m in range(3)]

    orig_step = piso.step

    def step_wrapped(prm, st, precond=None, dt=None):
        state["fresh"] = True
        state.pop("Rn", None)
        return orig_step(prm, st, precond, dt)

    monkeypatch.setattr(ops, "L", L_biased)
    monkeypatch.setattr(piso, "step", step_wrapped)
    r, nu, h = t_piso._tg_rate(16, nsteps=4)
    assert abs(r / (6 * nu * t_piso.s1(h)) - 1) > 2e-5


def test_solver_pin_catches_wrong_laplacian(monkeypatch):
    def helm_bad(prm, psi, dt, HbyA=None):
        h = prm.h

        def matvec(x):
            lap = ops.D([ops.G2(x, d, h) for d in range(3)], h)
            return psi * x / dt - dt * lap

        return matvec, psi / dt + 6.0 * dt / (h * h)

    monkeypatch.setattr(piso, "helmholtz", helm_bad)
    with pytest.raises(AssertionError):
        t_solve.test_pcg_uniform_psi_matches_fourier()


def test_rng_pin_catches_wrong_mixer_shift(monkeypatch):
    from oracle import ic

    from . import test_oracle_ic as t_ic

    def bad(seed, m):
        m = np.asarray(m, dtype=np.uint64)
        z = np.uint64(seed) + (m + np.uint64(1)) * ic.GOLDEN
        z = (z ^ (z >> np.uint64(31))) * ic.MIX1   # 30 in the published mixer
        z = (z ^ (z >> np.uint64(27))) * ic.MIX2
        return z ^ (z >> np.uint64(31))

    monkeypatch.setattr(ic, "splitmix64", bad)
    t_ic.test_uniform_moments()  # the statistical pins still pass
    with pytest.raises(AssertionError):
        t_ic.test_splitmix64_published_outputs()


def test_rng_pin_catches_zero_based_counter(monkeypatch):
    from oracle import ic

    from . import test_oracle_ic as t_ic
    orig = ic.splitmix64
    monkeypatch.setattr(ic, "splitmix64", lambda seed, m: orig(seed, np.asarray(m, dtype=np.uint64) - np.uint64(1)))
    with pytest.raises(AssertionError):
        t_ic.test_splitmix64_published_outputs()


def test_precond_pins_catch_a_wrong_jacobi_diagonal(monkeypatch):
    from oracle import unet

    from . import test_oracle_unet as t_unet
    monkeypatch.setattr(unet, "jacobi_diag", lambda psi, dt, h: psi / dt + 6.0 * dt / (h * h))
    with pytest.raises(AssertionError):
        t_unet.test_jacobi_diag_and_weight_channel_are_the_operators_entries()


def test_precond_pins_catch_a_target_without_the_jacobi_part(monkeypatch):
    from oracle import unet

    from . import test_oracle_unet as t_unet

    def bad_target(r, e, psi, dt, h):
        rho, d0 = unet.precond_scales(r, dt, h)
        return (e / (rho * d0))[None]

    monkeypatch.setattr(unet, "training_target", bad_target)
    with pytest.raises(AssertionError):
        t_unet.test_target_direction_solves_the_system(monkeypatch)


def test_les_pins_catch_uniform_filter_weights(monkeypatch):
    from oracle import les

    from . import test_oracle_les as t_les

    def uniform(m):
        return list(range(-m, m + 1)), np.full(2 * m + 1, 1.0 / (2 * m + 1))

    monkeypatch.setattr(les, "filter_weights", uniform)
    with pytest.raises(AssertionError):
        t_les.test_filter_transfer_function_is_the_dirichlet_closed_form(1)


def test_les_pins_catch_a_reynolds_filtered_stress(monkeypatch):
    from oracle import les

    from . import test_oracle_les as t_les

    def reynolds(rho, u, m):
        rb = les.box_filter(rho, m)
        ub = [les.box_filter(u[i], m) for i in range(3)]
        tau = [les.box_filter(rho * u[i] * u[j], m) - rb * ub[i] * ub[j] for i, j in les.PAIRS]
        return rb, ub, tau

    monkeypatch.setattr(les, "filtered_fields", reynolds)
    with pytest.raises(AssertionError):
        t_les.test_favre_stress_is_galilean_invariant()


def test_les_pins_catch_a_strain_without_the_half(monkeypatch):
    from oracle import les, ops

    from . import test_oracle_les as t_les

    def bad_strain(ut, h):
        g = [[ops.Gc(ut[i], j, h) for j in range(3)] for i in range(3)]
        return [g[i][j] + g[j][i] for i, j in les.PAIRS]

    monkeypatch.setattr(les, "strain", bad_strain)
    with pytest.raises(AssertionError):
        t_les.test_smagorinsky_tensor_of_a_shear_mode()


def test_two_fluid_pins_catch_a_trapezoidal_drag(monkeypatch):
    from oracle import twofluid

    from . import test_oracle_twofluid as t_tf

    def cn_drag(sig, mom, u, dt, tau):
        r = (1 - 0.5 * dt / tau) / (1 + 0.5 * dt / tau)
        return [u[m] + (mom[m] / sig - u[m]) * r for m in range(3)]

    monkeypatch.setattr(twofluid, "drag", cn_drag)
    with pytest.raises(AssertionError):
        t_tf.test_uniform_slip_relaxation_closed_form()


def test_two_fluid_pins_catch_a_flux_without_slip(monkeypatch):
    from oracle import ops, twofluid

    from . import test_oracle_twofluid as t_tf

    def no_slip(phi, rho, u, Y, V, h):
        F = [phi[d] * ops.I4(Y, d) for d in range(3)]
        return ops.D(F, h), [ops.D([F[d] * ops.I4(V[m], d) for d in range(3)], h) for m in range(3)]

    monkeypatch.setattr(twofluid, "dust_fluxes", no_slip)
    with pytest.raises(AssertionError):
        t_tf.test_first_order_agreement_with_the_equilibrium_model()


def test_isosurface_pins_catch_a_non_tiling_split(monkeypatch):
    from oracle import isosurface

    from . import test_oracle_isosurface as t_iso
    monkeypatch.setattr(isosurface, "TETS", [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7),
                                             (0, 2, 6, 4)])
    with pytest.raises(AssertionError):
        t_iso.test_planes_count_and_area_exact()


def test_isosurface_pins_catch_edge_points_from_either_end(monkeypatch):
    from oracle import isosurface

    from . import test_oracle_isosurface as t_iso

    def either_end(pa, fa, pb, fb, iso, a, b):
        t = (iso - fa) / (fb - fa)
        return tuple(pa[q] + t * (pb[q] - pa[q]) for q in range(3))

    monkeypatch.setattr(isosurface, "edge_point", either_end)
    with pytest.raises(AssertionError):
        t_iso.test_sphere_closed_and_second_order_area()
