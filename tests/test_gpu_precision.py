"""Mixed precision (FP32 fields and stencils; FP64-class Krylov inner products,
refinement residual and conserved totals): the error against the FP64
reference stated per quantity, and the horizon over which the turbulence
statistics named in Sec. 2 par. 1 (kinetic energy, enstrophy, Taylor
microscale; Fig. 1's density r.m.s.) stay within 1e-3.

Per step: one step from the same FP32-representable state through the mixed
GPU path and the FP64 oracle, for the 128^3 Fourier workload (r.m.s. Mach
0.5, k0 4, nu 0.002, one class Y 0.05, tau_p 0.1) and the 256^3 workload's
physics (barotropic, Mach 0.2, k0 8, nu 0.001) on a 128^3 box.  Every field's
relative L2 error and the relative error of every total and diagnostic are
printed as one "PRECISION ..." JSON line; bars: fields <= 1e-5, totals and
diagnostics <= 1e-5.

Horizon: the same spectral state (oracle initial field rounded to FP32) is
stepped by the mixed and the FP64 GPU paths (the FP64 path matches the oracle
to 1e-11 per step, test_gpu_step.py and test_gpu_fullsize.py): 200 steps of
the 128^3 Fourier workload (its stated length) and the first 80 steps of the
256^3 workload (the scheme itself becomes unstable on that workload near
t = 1.3, in FP64 and in mixed precision alike; see below).  The per-step relative differences of every diagnostic are
printed ("HORIZON ..." JSON lines: maximum, and the first step above 1e-3 if
any); bar: kinetic energy and enstrophy within 1e-3 over the whole horizon.
"""
import json

import numpy as np
import pytest

from oracle import diag as odiag
from oracle import piso
from paper_1404_0959_gb300.inputs import WORKLOADS

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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def f32_state(st):
    out = dict(st)
    for k in ("rho", "p", "T"):
        if st.get(k) is not None:
            out[k] = f32(st[k])
    for k in ("u", "phi", "Y"):
        out[k] = [f32(c) for c in st[k]]
    return out


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def relv(a, b):
    return abs(a - b) / abs(b) if b != 0 else abs(a)


def workload_prm(name, N, p_tol=1e-8):
    w = WORKLOADS[name]
    return piso.Params(N=N, closure=w["closure"], nu=w["nu"], tau_p=list(w["tau_p"]), Y0=list(w["Y0"]),
                       mach_rms=w["mach_rms"], k0=w["k0"], seed=w["seed"], p_tol=p_tol, p_maxit=1000)


def solver(fe, prm, precision):
    return fe.Solver([dict(N=prm.N, nu=prm.nu, tau_p=list(prm.tau_p), Y0=list(prm.Y0))], precision=precision,
                     closure=prm.closure, p_tol=prm.p_tol, p_maxit=prm.p_maxit)


GPU_DIAG = ("ke", "enstrophy", "taylor", "rho_rms")


@pytest.mark.parametrize("name", ["hit128f", "hit256"])
def test_per_quantity_step_error_against_the_oracle(fe, name):
    N = 128
    prm = workload_prm(name, N)
    fourier = prm.closure == piso.FOURIER
    st = f32_state(piso.initial_state(prm))
    ref, rinfo = piso.step(prm, st)
    s = solver(fe, prm, fe.FE_FP32_MIXED)
    s.load_state(0, st)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    d = s.diagnostics(0)
    s.close()
    err = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"])}
    err["u"] = max(rel(got["u"][m], ref["u"][m]) for m in range(3))
    err["phi"] = max(rel(got["phi"][m], ref["phi"][m]) for m in range(3))
    err["Y"] = max(rel(got["Y"][j], ref["Y"][j]) for j in range(len(ref["Y"])))
    if fourier:
        err["T"] = rel(got["T"], ref["T"])
    tot = piso.totals(prm, ref)
    err["mass"] = relv(d["mass"], tot["mass"])
    err["dust_mass"] = relv(d["dust_mass"][0], tot["dust"][0])
    err["energy"] = relv(d["energy"], tot["energy"])
    r = odiag.diagnostics(ref["rho"], ref["u"], prm.h)
    for k in GPU_DIAG:
        err[k] = relv(d[k], r[k])
    err["dt"] = relv(info[0]["dt"], rinfo["dt"])
    print("PRECISION " + json.dumps({"workload": name, "N": N, "iters": info[0]["iters"],
                                     "oracle_iters": rinfo["iters"],
                                     "rel_err": {k: float("%.3g" % v) for k, v in err.items()}}))
    assert max(info[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert max(err.values()) < 1e-5, err


def _horizon(fe, name, N, steps):
    prm = workload_prm(name, N)
    st = f32_state(piso.initial_state(prm))
    s64 = solver(fe, prm, fe.FE_FP64)
    s32 = solver(fe, prm, fe.FE_FP32_MIXED)
    s64.load_state(0, st)
    s32.load_state(0, st)
    s32.use_graphs(True)
    keys = GPU_DIAG + ("mass", "dust_mass", "energy")
    worst = {k: 0.0 for k in keys}
    first = {k: None for k in keys}
    hist = []
    for n in range(1, steps + 1):
        c64, _ = s64.step(1)
        c32, _ = s32.step(1)
        assert c64 == fe.FE_OK and c32 == fe.FE_OK, (n, fe.fe_strerror(c64), fe.fe_strerror(c32))
        a, b = s32.diagnostics(0), s64.diagnostics(0)
        row = {}
        for k in keys:
            va = a[k][0] if k == "dust_mass" else a[k]
            vb = b[k][0] if k == "dust_mass" else b[k]
            e = relv(va, vb)
            row[k] = e
            worst[k] = max(worst[k], e)
            if first[k] is None and e > 1e-3:
                first[k] = n
        hist.append(row)
    t = b["t"]
    s64.close()
    s32.close()
    marks = [s for s in (1, 10, 50, 80, 100, 200, 300, 400, 500) if s <= steps]
    print("HORIZON " + json.dumps({"workload": name, "N": N, "steps": steps, "t_end": t,
                                   "max_rel_diff": {k: float("%.3g" % v) for k, v in worst.items()},
                                   "first_step_above_1e-3": first,
                                   "ke_at": {m: float("%.3g" % hist[m - 1]["ke"]) for m in marks},
                                   "enstrophy_at": {m: float("%.3g" % hist[m - 1]["enstrophy"]) for m in marks}}))
    return worst


def test_mixed_history_horizon_128_fourier_200_steps(fe):
    w = _horizon(fe, "hit128f", 128, WORKLOADS["hit128f"]["steps"])
    assert w["ke"] < 1e-3 and w["enstrophy"] < 1e-3, w


# The scheme as read (fourth-order central interpolation with no added dissipation) does not carry
# the 256^3 barotropic workload past t ~ 1.3: grid-scale density oscillations grow and the step turns
# non-finite at step 103 in FP64 and step 91 in mixed precision (the symmetric and the transonic
# pressure equation, two or three correctors, and a pressure-balanced start alike).  The horizon is
# therefore measured over the 80 steps (t ~ 1.0) before that.
HIT256_STABLE_STEPS = 80


def test_mixed_history_horizon_256_barotropic_stable_range(fe):
    w = _horizon(fe, "hit256", 256, HIT256_STABLE_STEPS)
    assert w["ke"] < 1e-3 and w["enstrophy"] < 1e-3, w
