"""GPU parity of fe_solve_pressure, fe_init_state, fe_diagnostics and
fe_q_criterion against the FP64 oracle (and the closed-form solve)."""
import math

import numpy as np
import pytest

from oracle import diag as odiag
from oracle import ic as oic
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


@pytest.mark.parametrize("N", [16, 40])
def test_solve_pressure_matches_oracle_pcg(fe, N):
    import torch
    rho, u, Y, T = random_fields(N, 1, False, seed=2, noise=0.02)
    prm = piso.Params(N=N)
    st = piso.make_state(prm, rho, u, Y)
    psi = st["rho"] / (prm.gamma * st["p"])
    dt = 0.07
    matvec, dg = piso.helmholtz(prm, psi, dt)
    b = random_vector(N, 3)
    x_ref, it_ref, _, true_ref = krylov.pcg(matvec, b, dg, 1e-11, 500)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, rho, u, Y)
    code, x, info = s.solve_pressure(0, torch.tensor(b, device="cuda"), dt, 1e-11, 500)
    assert code == fe.FE_OK
    assert abs(info.iters - it_ref) <= 1
    assert info.rel_res_true < 1e-11
    assert rel(x.cpu().numpy(), x_ref) < 1e-10
    s.close()


def test_solve_pressure_closed_form_uniform_psi(fe):
    import torch
    N = 32
    ones = np.ones((N, N, N))
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, 1.1 * ones, [0 * ones] * 3, [0.01 * ones])
    psi0 = 1.1 / (1.1 ** 1.4)
    dt = 0.2
    b = random_vector(N, 4)
    code, x, info = s.solve_pressure(0, torch.tensor(b, device="cuda"), dt, 1e-13, 800)
    assert code == fe.FE_OK
    h = 2 * math.pi / N
    kk = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    lam = psi0 / dt + 0.5 * dt * sum(4 * np.sin(k * h / 2) ** 2 / h ** 2 for k in (kx, ky, kz))
    xe = np.real(np.fft.ifftn(np.fft.fftn(b) / lam))
    assert rel(x.cpu().numpy(), xe) < 1e-11
    s.close()


def test_solve_pressure_not_converged_reported(fe):
    import torch
    N = 16
    rho, u, Y, T = random_fields(N, 1, False, seed=2)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, rho, u, Y)
    code, x, info = s.solve_pressure(0, torch.tensor(random_vector(N, 1), device="cuda"), 0.5, 1e-14, 2)
    assert code == fe.FE_ERR_NOT_CONVERGED
    assert info.iters == 2
    s.close()


@pytest.mark.parametrize("N,k0,mach,seed", [(32, 4.0, 0.2, 0), (48, 4.0, 0.5, 7), (24, 3.0, 0.3, 11)])
def test_spectral_initial_state(fe, N, k0, mach, seed):
    ref = oic.spectral_velocity(N, k0, mach, seed)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01], mach_rms=mach, k0=k0, seed=seed)])
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    st = s.get_state(0)
    for d in range(3):
        assert rel(st["u"][d], ref[d]) < 1e-12
    assert np.all(st["rho"] == 1.0)
    assert np.all(st["Y"][0] == 0.01)
    prm = piso.Params(N=N)
    ost = piso.make_state(prm, np.ones((N, N, N)), ref, [np.full((N, N, N), 0.01)])
    for d in range(3):
        assert rel(st["phi"][d], ost["phi"][d]) < 1e-12
    s.close()


def test_diagnostics_and_spectrum(fe):
    N = 32
    rho, u, Y, T = random_fields(N, 2, True, seed=6)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05, 0.1], Y0=[0.01, 0.02])], closure=fe.FE_FOURIER)
    s.set_state(0, rho, u, Y, T)
    h = 2 * math.pi / N
    nb = 30
    d = s.diagnostics(0, nbins=nb)
    ref = odiag.diagnostics(rho, u, h, nbins=nb)
    for k in ("ke", "ke_u", "enstrophy", "taylor", "rho_rms"):
        assert abs(d[k] - ref[k]) <= 1e-12 * abs(ref[k]), k
    np.testing.assert_allclose(d["spectrum"], ref["spectrum"], rtol=1e-11, atol=1e-16)
    prm = piso.Params(N=N, closure=piso.FOURIER, tau_p=[0.05, 0.1], Y0=[0.01, 0.02])
    tot = piso.totals(prm, piso.make_state(prm, rho, u, Y, T))
    assert abs(d["mass"] - tot["mass"]) <= 1e-13 * tot["mass"]
    assert abs(d["energy"] - tot["energy"]) <= 1e-13 * tot["energy"]
    for j in range(2):
        assert abs(d["dust_mass"][j] - tot["dust"][j]) <= 1e-13 * tot["dust"][j]
    s.close()


def test_q_criterion(fe):
    N = 24
    rho, u, Y, T = random_fields(N, 1, False, seed=8)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, rho, u, Y)
    q = s.q_criterion(0).cpu().numpy()
    ref = odiag.q_criterion(u, 2 * math.pi / N)
    assert rel(q, ref) < 1e-13
    s.close()
