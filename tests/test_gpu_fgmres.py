"""Flexible GMRES(20) pressure solver (FE_FGMRES_LEARNED) against the FP64
oracle's flexible GMRES: the solve alone on the transonic (non-symmetric)
operator, PISO steps with either operator in FP64 and in mixed precision,
and convergence with an arbitrary network supplying the directions.

Bars: FP64 solves agree with the oracle's flexible GMRES (same restart
length, Jacobi directions) within one iteration and 1e-9 in x at tolerance
1e-11; FP64 steps within 1e-11 per field of the oracle step with the same
solver; mixed precision within 1e-5 of the oracle from the same FP32 state.
"""
import numpy as np
import pytest

from oracle import krylov, piso
from paper_1404_0959_gb300.inputs import random_fields, random_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1404_0959_gb300 import build
    build.build()
    from paper_1404_0959_gb300 import fe as fe_mod
    return fe_mod


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("N", [16, 24])
def test_transonic_solve_matches_oracle_fgmres(fe, N):
    """fe_solve_pressure with Jacobi directions (no network loaded): the
    operator uses psi of the state and HbyA = u."""
    import torch
    rho, u, Y, T = random_fields(N, 1, False, seed=3, noise=0.02, mach=0.3)
    prm = piso.Params(N=N, transonic=True)
    st = piso.make_state(prm, rho, u, Y)
    psi = st["rho"] / (prm.gamma * st["p"])
    dt = 0.08
    matvec, dg = piso.helmholtz(prm, psi, dt, st["u"])
    b = random_vector(N, 5)
    x_ref, it_ref, _, _ = krylov.fgmres(matvec, b, None, dg, 1e-11, 500, m=20)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], solver=fe.FE_FGMRES_LEARNED, transonic=True)
    s.set_state(0, rho, u, Y)
    code, x, info = s.solve_pressure(0, torch.tensor(b, device="cuda"), dt, 1e-11, 500)
    s.close()
    assert code == fe.FE_OK, fe.fe_strerror(code)
    assert abs(info.iters - it_ref) <= 1, (info.iters, it_ref)
    assert info.rel_res_true <= 1e-11 * 1.01
    assert rel(x.cpu().numpy(), x_ref) < 1e-9


def _step_pair(fe, N, transonic, precision, p_tol, seed=1):
    rho, u, Y, T = random_fields(N, 1, False, seed=seed, noise=0.02, mach=0.3)
    prm = piso.Params(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01], transonic=transonic, fgmres=True, p_tol=p_tol)
    st = piso.make_state(prm, rho, u, Y)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=precision,
                  solver=fe.FE_FGMRES_LEARNED, transonic=transonic, p_tol=p_tol)
    if precision == fe.FE_FP64:
        s.set_state(0, rho, u, Y)
    else:  # the oracle steps the FP32-rounded state
        st = {k: ([f32(c) for c in v] if isinstance(v, list) else (f32(v) if isinstance(v, np.ndarray) else v))
              for k, v in st.items()}
        s.load_state(0, st)
    ref, info = piso.step(prm, st)
    code, ginf = s.step(1)
    got = s.get_state(0)
    s.close()
    assert code == fe.FE_OK, fe.fe_strerror(code)
    errs = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"]), "Y": rel(got["Y"][0], ref["Y"][0])}
    for d in range(3):
        errs["u%d" % d] = rel(got["u"][d], ref["u"][d])
        errs["phi%d" % d] = rel(got["phi"][d], ref["phi"][d])
    return errs, ginf[0], info


@pytest.mark.parametrize("transonic", [True, False])
def test_fp64_step_matches_oracle(fe, transonic):
    errs, ginf, info = _step_pair(fe, 16, transonic, fe.FE_FP64, 1e-10)
    assert max(errs.values()) <= 1e-11, errs
    assert all(abs(a - b) <= 1 for a, b in zip(ginf["iters"], info["iters"])), (ginf["iters"], info["iters"])
    assert max(ginf["rel_res"]) <= 1e-10 * 1.01


def test_mixed_step_matches_oracle(fe):
    errs, ginf, _ = _step_pair(fe, 24, True, fe.FE_FP32_MIXED, 1e-8)
    assert max(errs.values()) <= 1e-5, errs
    assert max(ginf["rel_res"]) <= 1e-8 * 1.01


def test_converges_with_any_network(fe):
    """Random (untrained) network directions: flexible GMRES still reaches the
    tolerance on the transonic operator, and the solution is the oracle's."""
    import torch
    from paper_1404_0959_gb300 import learned
    N = 16
    rho, u, Y, T = random_fields(N, 1, False, seed=4, noise=0.02, mach=0.3)
    prm = piso.Params(N=N, transonic=True)
    st = piso.make_state(prm, rho, u, Y)
    psi = st["rho"] / (prm.gamma * st["p"])
    dt = 0.08
    matvec, dg = piso.helmholtz(prm, psi, dt, st["u"])
    b = random_vector(N, 6)
    x_ref, _, _, _ = krylov.bicgstab(matvec, b, dg, 1e-13, 500)
    for every in (1, 0):
        s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], solver=fe.FE_FGMRES_LEARNED,
                      transonic=True, learned_every=every)
        s.set_state(0, rho, u, Y)
        fe.fe_load_preconditioner(s.ctx, learned.he_init(3, zero_last=False))
        code, x, info = s.solve_pressure(0, torch.tensor(b, device="cuda"), dt, 1e-10, 500)
        s.close()
        assert code == fe.FE_OK, fe.fe_strerror(code)
        assert info.rel_res_true <= 1e-10 * 1.01
        assert rel(x.cpu().numpy(), x_ref) < 1e-8
