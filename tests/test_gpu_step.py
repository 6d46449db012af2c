"""GPU parity of the PISO step (through the C ABI) against the FP64 oracle.

Inputs come from the seeded generators in paper_1404_0959_gb300.inputs and
are given to both sides.  FP64 bar: relative L2 error <= 1e-11 per field and
per step (both sides run the same Krylov iteration to the same tolerance, so
they differ only by rounding order).  Sizes span several tiles and ragged
tile edges (N not a multiple of 32 in x).
"""
import numpy as np
import pytest

from oracle import piso
from paper_1404_0959_gb300.inputs import random_fields

pytestmark = pytest.mark.gpu

TOL64 = 1e-11


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
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / (nb if nb > 0 else 1.0)


def compare(got, ref, tol, fourier=False):
    errs = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"])}
    for d in range(3):
        errs["u%d" % d] = rel(got["u"][d], ref["u"][d])
        errs["phi%d" % d] = rel(got["phi"][d], ref["phi"][d])
    for j in range(len(ref["Y"])):
        errs["Y%d" % j] = rel(got["Y"][j], ref["Y"][j])
    if fourier:
        errs["T"] = rel(got["T"], ref["T"])
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (bad, errs)
    return errs


def run_pair(fe, N, nsteps=1, closure=0, tau_p=(0.05,), Y0=(0.01,), nu=0.005, transonic=False, seed=1,
             noise=0.02, mach=0.3, n_corr=2, p_tol=1e-10):
    fourier = closure == piso.FOURIER
    rho, u, Y, T = random_fields(N, len(tau_p), fourier, seed=seed, mach=mach, noise=noise)
    prm = piso.Params(N=N, closure=closure, nu=nu, tau_p=list(tau_p), Y0=list(Y0), transonic=transonic,
                      n_corr=n_corr, p_tol=p_tol)
    st = piso.make_state(prm, rho, u, Y, T)
    solver = fe.FE_BICGSTAB_JACOBI if transonic else fe.FE_PCG_JACOBI
    s = fe.Solver([dict(N=N, nu=nu, tau_p=list(tau_p), Y0=list(Y0))], closure=closure, transonic=transonic,
                  solver=solver, n_corr=n_corr, p_tol=p_tol)
    s.set_state(0, rho, u, Y, T)
    init = s.get_state(0)
    compare(init, st, 1e-14, fourier)  # derived p and phi agree before stepping
    infos = []
    for _ in range(nsteps):
        st, info = piso.step(prm, st)
        code, ginf = s.step(1)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        infos.append((info, ginf[0]))
        assert abs(ginf[0]["dt"] - info["dt"]) <= 1e-13 * info["dt"]
    got = s.get_state(0)
    s.close()
    return got, st, infos


@pytest.mark.parametrize("N", [16, 24, 40])
def test_one_step_barotropic(fe, N):
    got, ref, infos = run_pair(fe, N)
    compare(got, ref, TOL64)
    info, ginf = infos[0]
    assert all(abs(a - b) <= 1 for a, b in zip(ginf["iters"], info["iters"]))
    assert max(ginf["rel_res"]) < 1e-10


def test_one_step_fourier_three_classes(fe):
    got, ref, _ = run_pair(fe, 24, closure=piso.FOURIER, tau_p=(0.02, 0.1, 0.3), Y0=(0.02, 0.02, 0.02),
                           nu=0.002, mach=0.5)
    compare(got, ref, TOL64, fourier=True)


def test_transonic_bicgstab(fe):
    got, ref, _ = run_pair(fe, 16, transonic=True)
    compare(got, ref, TOL64)


def test_five_steps_hit32_physics(fe):
    got, ref, infos = run_pair(fe, 32, nsteps=5, noise=0.0, mach=0.2)
    compare(got, ref, 5 * TOL64)


def test_three_correctors_and_one_corrector(fe):
    for nc in (1, 3):
        got, ref, _ = run_pair(fe, 16, n_corr=nc, seed=3)
        compare(got, ref, TOL64)


def test_minimum_grid(fe):
    got, ref, _ = run_pair(fe, 8, seed=4)
    compare(got, ref, TOL64)


def test_uniform_state_zero_rhs(fe):
    N = 16
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], dt_max=0.1)
    ones = np.ones((N, N, N))
    s.set_state(0, 1.3 * ones, [0.1 * ones, 0.05 * ones, 0 * ones], [0.01 * ones])
    code, info = s.step(1)
    assert code == fe.FE_OK
    assert info[0]["iters"] == [0, 0]
    st = s.get_state(0)
    assert np.max(np.abs(st["rho"] - 1.3)) < 1e-14
    assert np.max(np.abs(st["u"][0] - 0.1)) < 1e-15
    assert np.max(np.abs(st["Y"][0] - 0.01)) < 1e-16
    s.close()


def test_conservation_on_gpu(fe):
    N = 32
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    rho, u, Y, T = random_fields(N, 1, False, seed=9, noise=0.02)
    s.set_state(0, rho, u, Y)
    d0 = s.diagnostics(0)
    code, _ = s.step(3)
    assert code == fe.FE_OK
    d1 = s.diagnostics(0)
    assert abs(d1["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d1["dust_mass"][0] - d0["dust_mass"][0]) <= 1e-13 * d0["dust_mass"][0]
    s.close()


def test_batched_field_copies(fe):
    # fe_set_fields / fe_get_fields move the same bytes as one call per field,
    # from host and from device memory; a bad id copies nothing
    import torch
    N = 24
    rho, u, Y, _ = random_fields(N, 1, False, seed=21, noise=0.02)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, rho, u, Y)
    ids = [fe.FE_RHO, fe.FE_UX, fe.FE_UY, fe.FE_UZ, fe.FE_P, fe.FE_PHIX, fe.FE_PHIY, fe.FE_PHIZ, fe.FE_Y0]
    single = {f: s.get_field(0, f) for f in ids}
    host = [np.empty((N, N, N)) for _ in ids]
    fe.fe_get_fields(s.ctx, 0, ids, [h.ctypes.data for h in host], 0)
    for f, h in zip(ids, host):
        assert np.array_equal(h, single[f])
    # write scaled copies back from device memory, read them again
    dev = [torch.tensor(2.0 * h, device="cuda") for h in host]
    fe.fe_set_fields(s.ctx, 0, ids, [d.data_ptr() for d in dev], 1)
    for f, h in zip(ids, host):
        assert np.array_equal(s.get_field(0, f), 2.0 * h)
    before = s.get_field(0, fe.FE_RHO)
    with pytest.raises(fe.FeError):
        fe.fe_set_fields(s.ctx, 0, [fe.FE_RHO, 999], [dev[0].data_ptr(), dev[1].data_ptr()], 1)
    assert np.array_equal(s.get_field(0, fe.FE_RHO), before)
    s.close()


@pytest.mark.parametrize("N,prec", [(24, 0), (32, 1), (21, 1)])
def test_batched_copies_through_page_locked_host_memory(fe, N, prec):
    # page-locked host buffers (the end-to-end benchmark's path), both precisions, an odd size
    import torch
    rho, u, Y, _ = random_fields(N, 1, False, seed=22, noise=0.02)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=prec)
    s.set_state(0, rho, u, Y)
    ids = [fe.FE_RHO, fe.FE_UX, fe.FE_UY, fe.FE_UZ, fe.FE_P, fe.FE_PHIX, fe.FE_PHIY, fe.FE_PHIZ, fe.FE_Y0]
    single = {f: s.get_field(0, f) for f in ids}
    dt = torch.float64 if prec == 0 else torch.float32
    pinned = [torch.empty((N, N, N), dtype=dt, pin_memory=True) for _ in ids]
    fe.fe_get_fields(s.ctx, 0, ids, [h.data_ptr() for h in pinned], 0)
    for f, h in zip(ids, pinned):
        assert np.array_equal(h.numpy(), single[f])
    for h in pinned:
        h.mul_(3.0)
    fe.fe_set_fields(s.ctx, 0, ids, [h.data_ptr() for h in pinned], 0)
    for f, h in zip(ids, pinned):
        assert np.array_equal(s.get_field(0, f), h.numpy())
    s.close()
