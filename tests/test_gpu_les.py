"""A-priori LES analysis on the GPU (fe_les_apriori) against the oracle
(oracle/les.py: trapezoidal top-hat filter of width 2 m h, Favre sub-grid
stress, Smagorinsky model slot, box statistics; the paper's Sec. 1 and 2 name
LES and a-priori tests of the DNS database but no filter or model).

FP64: the filtered density, Favre velocity and the six stress components
element by element within 1e-12 (relative L2), every statistic within 1e-11,
on grids that are and are not multiples of the launch chunk (N = 16, 24, 30)
for m = 1, 2, 3, and on a 128^3 spectral turbulence field.  FP32 fields:
rho_bar and u~ within 1e-6; the stress, a difference of two filtered
products, within 1e-6 of the scale of those products; statistics within 1e-4.
"""
import numpy as np
import pytest

from oracle import les, piso
from paper_1404_0959_gb300.inputs import WORKLOADS, random_fields

pytestmark = pytest.mark.gpu

STATS = ("delta", "k_sgs", "pi_sgs", "cs2_opt", "corr", "pi_model")


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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gpu_les(fe, rho, u, m, cs, precision):
    import torch
    N = rho.shape[0]
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=precision)
    s.set_state(0, rho, u, [0.01 * np.ones_like(rho)])
    dt = torch.float64 if precision == fe.FE_FP64 else torch.float32
    out = torch.full((10, N, N, N), float("nan"), dtype=dt, device="cuda")
    st = fe.fe_les_apriori(s.ctx, 0, m, cs, out.data_ptr())
    st2 = fe.fe_les_apriori(s.ctx, 0, m, cs)  # second call, no field output: the same statistics
    f = out.double().cpu().numpy()
    s.close()
    assert st2 == st
    return st, f


def compare(st, f, rho, u, N, m, cs, tol_f, tol_s, tau_scale_tol=None):
    h = 2 * np.pi / N
    rb, ut, tau = les.filtered_fields(rho, u, m)
    want = les.apriori(rho, u, h, m, cs)
    errs = {"rho_bar": rel(f[0], rb)}
    for i in range(3):
        errs["u%d" % i] = rel(f[1 + i], ut[i])
    if tau_scale_tol is None:
        for q in range(6):
            errs["tau%d" % q] = rel(f[4 + q], tau[q])
        assert max(errs.values()) < tol_f, errs
    else:
        assert max(errs.values()) < tol_f, errs
        scale = np.linalg.norm(les.box_filter(rho * u[0] * u[0], m))
        for q in range(6):
            e = float(np.linalg.norm(f[4 + q] - tau[q]) / scale)
            errs["tau%d" % q] = e
            assert e < tau_scale_tol, errs
    serr = {k: abs(st[k] - want[k]) / max(abs(want[k]), 1e-300) for k in STATS}
    assert max(serr.values()) < tol_s, (serr, st, want)
    return errs, serr


@pytest.mark.parametrize("N", [16, 24, 30])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_fp64_les_matches_oracle(fe, N, m):
    rho, u, _, _ = random_fields(N, 0, False, seed=30 + N + m, drho=0.08, noise=0.05)
    st, f = gpu_les(fe, rho, u, m, 0.17, fe.FE_FP64)
    compare(st, f, rho, u, N, m, 0.17, 1e-12, 1e-11)


def test_fp64_les_on_spectral_turbulence_at_128(fe):
    w = WORKLOADS["hit128f"]
    N, m = 128, 2
    prm = piso.Params(N=N, closure=w["closure"], nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], mach_rms=w["mach_rms"],
                      k0=w["k0"], seed=0)
    st0 = piso.initial_state(prm)
    rho = 1.0 + 0.02 * st0["u"][0]  # a variable density so that Favre and plain filtering differ
    st, f = gpu_les(fe, rho, st0["u"], m, 0.17, fe.FE_FP64)
    errs, serr = compare(st, f, rho, st0["u"], N, m, 0.17, 1e-12, 1e-11)
    print("128^3 a-priori statistics:", {k: "%.6e" % st[k] for k in STATS}, "max field error %.1e stat %.1e"
          % (max(errs.values()), max(serr.values())))


@pytest.mark.parametrize("N,m", [(24, 1), (32, 2)])
def test_fp32_les_matches_oracle(fe, N, m):
    rho, u, _, _ = random_fields(N, 0, False, seed=7 + N, drho=0.08, noise=0.05)
    rho, u = f32(rho), [f32(c) for c in u]
    st, f = gpu_les(fe, rho, u, m, 0.17, fe.FE_FP32_MIXED)
    errs, serr = compare(st, f, rho, u, N, m, 0.17, 1e-6, 1e-4, tau_scale_tol=1e-6)
    print("FP32 N=%d m=%d: field errors %.1e, stat errors %.1e" % (N, m, max(errs.values()), max(serr.values())))


def test_les_rejects_bad_widths(fe):
    N = 16
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    for m in (0, fe.FE_LES_MAX_M + 1, 8):  # 2 m + 1 > N for m = 8 at N = 16
        with pytest.raises(fe.FeError):
            fe.fe_les_apriori(s.ctx, 0, m, 0.17)
    s.close()
