"""Mixed precision: FP32 fields and stencils, FP64 Krylov dot products, FP64
iterative refinement of the pressure solve and FP64 conserved totals.

Bars: per-step fields within 1e-5 (relative L2) of the FP64 oracle started
from the same (FP32-representable) state; kinetic-energy and enstrophy
histories within 1e-3 over 20 steps at 32^3; the FP64 pressure residual
meets the requested tolerance.  At the benchmark size (256^3, bench launch
configuration) the mixed step is compared with the FP64 GPU step and checked
for conservation, residuals and translation invariance.
"""
import math

import numpy as np
import pytest

from oracle import diag as odiag
from oracle import krylov, piso
from paper_1404_0959_gb300.inputs import WORKLOADS, random_fields, random_vector

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def fe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1404_0959_gb300 import build
    build.build()
    from paper_1404_0959_gb300 import fe as fe_mod
    return fe_mod


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0)


def state_errors(got, ref, fourier=False):
    e = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"])}
    for d in range(3):
        e["u%d" % d] = rel(got["u"][d], ref["u"][d])
        e["phi%d" % d] = rel(got["phi"][d], ref["phi"][d])
    for j in range(len(ref["Y"])):
        e["Y%d" % j] = rel(got["Y"][j], ref["Y"][j])
    if fourier:
        e["T"] = rel(got["T"], ref["T"])
    return e


def f32_state(st):
    """Round a state to FP32 values (kept as float64 arrays for the oracle)."""
    out = dict(st)
    for k in ("rho", "p", "T"):
        if st.get(k) is not None:
            out[k] = f32(st[k])
    for k in ("u", "phi", "Y"):
        out[k] = [f32(c) for c in st[k]]
    return out


def mixed_pair(fe, N, closure=0, tau_p=(0.05,), Y0=(0.01,), nu=0.005, mach=0.3, seed=1, p_tol=1e-8, noise=0.02):
    """Oracle state (p and phi derived by the oracle) rounded to FP32, loaded into an FP32 context."""
    fourier = closure == piso.FOURIER
    rho, u, Y, T = random_fields(N, len(tau_p), fourier, seed=seed, mach=mach, noise=noise)
    prm = piso.Params(N=N, closure=closure, nu=nu, tau_p=list(tau_p), Y0=list(Y0), p_tol=p_tol)
    st = f32_state(piso.make_state(prm, f32(rho), [f32(c) for c in u], [f32(y) for y in Y],
                                   f32(T) if fourier else None))
    s = fe.Solver([dict(N=N, nu=nu, tau_p=list(tau_p), Y0=list(Y0))], precision=fe.FE_FP32_MIXED, closure=closure,
                  p_tol=p_tol)
    s.load_state(0, st)
    return s, prm, st


# N = 30 is not a multiple of the 16-byte chunk: every stage, the right-hand side that starts the
# refined solve and the refinement boundary run their z-marching kernels
@pytest.mark.parametrize("N", [24, 30, 40])
def test_mixed_one_step_vs_fp64_oracle(fe, N):
    s, prm, st = mixed_pair(fe, N)
    ref, info = piso.step(prm, st)
    code, ginf = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    assert max(ginf[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    e = state_errors(s.get_state(0), ref)
    assert max(e.values()) < TOL32, e
    s.close()


def test_mixed_fourier_three_classes(fe):
    s, prm, st = mixed_pair(fe, 24, closure=piso.FOURIER, tau_p=(0.02, 0.1, 0.3), Y0=(0.02, 0.02, 0.02), nu=0.002,
                            mach=0.5)
    ref, _ = piso.step(prm, st)
    code, _ = s.step(1)
    assert code == fe.FE_OK
    e = state_errors(s.get_state(0), ref, fourier=True)
    assert max(e.values()) < TOL32, e
    s.close()


@pytest.mark.parametrize("N,solver", [(32, "jacobi"), (32, "poly"), (64, "poly")])
def test_mixed_histories_20_steps(fe, N, solver):
    """KE and enstrophy histories of the hit32 physics within 1e-3 over 20 steps, with Jacobi-PCG and
    with the Neumann-polynomial CG (z-marched at 32^3, plane-streamed at 64^3)."""
    w = WORKLOADS["hit32"]
    from oracle import ic as oic
    u0 = [f32(c) for c in oic.spectral_velocity(N, w["k0"], w["mach_rms"], 0)]
    ones = np.ones((N, N, N))
    prm = piso.Params(N=N, nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], p_tol=1e-8)
    s = fe.Solver([dict(N=N, nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"])], precision=fe.FE_FP32_MIXED, p_tol=1e-8,
                  solver=fe.FE_PCG_POLY if solver == "poly" else fe.FE_PCG_JACOBI)
    st = f32_state(piso.make_state(prm, ones, u0, [f32(0.01 * ones)]))
    s.load_state(0, st)
    h = 2 * math.pi / N
    worst_ke = worst_om = 0.0
    for n in range(20):
        st, _ = piso.step(prm, st)
        code, _ = s.step(1)
        assert code == fe.FE_OK
        d = s.diagnostics(0)
        r = odiag.diagnostics(st["rho"], st["u"], h)
        worst_ke = max(worst_ke, abs(d["ke"] - r["ke"]) / r["ke"])
        worst_om = max(worst_om, abs(d["enstrophy"] - r["enstrophy"]) / r["enstrophy"])
    assert worst_ke < 1e-3 and worst_om < 1e-3, (worst_ke, worst_om)
    s.close()


def test_mixed_solve_reaches_fp64_residual(fe):
    import torch
    N = 32
    rho, u, Y, T = random_fields(N, 1, False, seed=4, noise=0.02)
    prm0 = piso.Params(N=N)
    st = f32_state(piso.make_state(prm0, f32(rho), [f32(c) for c in u], [f32(Y[0])]))
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED)
    s.load_state(0, st)
    # psi as the GPU forms it: FP32 rho / (FP32 gamma * FP32 p), rounded to FP32
    psi = f32(np.float32(st["rho"]) / (np.float32(1.4) * np.float32(st["p"])))
    dt = 0.08
    b = f32(random_vector(N, 5))
    for tol in (1e-8, 1e-10):
        code, x, info = s.solve_pressure(0, torch.tensor(b, dtype=torch.float32, device="cuda"), dt, tol, 500)
        assert code == fe.FE_OK
        assert info.rel_res_true <= tol
        prm = piso.Params(N=N)
        matvec, dg = piso.helmholtz(prm, psi, dt)
        xr, _, _, _ = krylov.pcg(matvec, b, dg, 1e-13, 500)
        # x is returned in FP32: agreement to FP32 rounding of the converged solution
        assert rel(x.cpu().numpy(), xr) < 1e-6
    s.close()


def _bench_solver(fe, precision, seed=0):
    w = WORKLOADS["hit256"]
    s = fe.Solver([dict(N=w["N"], nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], mach_rms=w["mach_rms"], k0=w["k0"],
                        seed=seed)], precision=precision, p_tol=w["p_tol"], p_maxit=1000)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    return s


def test_full_size_mixed_vs_fp64_gpu_and_properties(fe):
    """256^3, bench configuration: one mixed step vs one FP64 step from the same
    initial field; mass and dust conservation; FP64 residuals <= 1e-8."""
    s64 = _bench_solver(fe, fe.FE_FP64)
    s32 = _bench_solver(fe, fe.FE_FP32_MIXED)
    d0 = s32.diagnostics(0)
    c64, i64 = s64.step(1)
    c32, i32 = s32.step(1)
    assert c64 == fe.FE_OK and c32 == fe.FE_OK
    assert max(i32[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert max(i64[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    a = s32.get_state(0)
    b = s64.get_state(0)
    e = state_errors(a, b)
    assert max(e.values()) < TOL32, e
    d1 = s32.diagnostics(0)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-6 * d0["mass"]
    assert abs(d1["dust_mass"][0] - d0["dust_mass"][0]) <= 1e-6 * d0["dust_mass"][0]
    s64.close()
    s32.close()


def test_full_size_translation_invariance(fe):
    """Shifting the 256^3 input by (3, 5, 7) cells shifts the output: catches tile
    and wrap indexing errors at the benchmark size (reduction order aside)."""
    s1 = _bench_solver(fe, fe.FE_FP32_MIXED)
    st = s1.get_state(0)
    sh = (7, 5, 3)  # numpy axes (z, y, x)
    s2 = fe.Solver([dict(N=256, nu=0.001, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED, p_tol=1e-8,
                   p_maxit=1000)
    s2.set_state(0, np.roll(st["rho"], sh, (0, 1, 2)), [np.roll(c, sh, (0, 1, 2)) for c in st["u"]],
                 [np.roll(st["Y"][0], sh, (0, 1, 2))])
    c1, _ = s1.step(1)
    c2, _ = s2.step(1)
    assert c1 == fe.FE_OK and c2 == fe.FE_OK
    a = s1.get_state(0)
    b = s2.get_state(0)
    for k in ("rho", "p"):
        assert rel(np.roll(a[k], sh, (0, 1, 2)), b[k].astype(np.float64)) < TOL32
    for d in range(3):
        assert rel(np.roll(a["u"][d], sh, (0, 1, 2)), b["u"][d].astype(np.float64)) < TOL32
    s1.close()
    s2.close()
