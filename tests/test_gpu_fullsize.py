"""Full benchmark size (256^3 isotropic turbulence, barotropic, M 0.2, k0 8,
nu 0.001, one dust class, pressure residual 1e-8) against the FP64 oracle.

The oracle's step at this size takes minutes, so its result is stored:
tests/golden/hit256_step.json, written by tests/golden/make_golden_hit256.py
from the oracle alone (the oracle's spectral initial state rounded to FP32, one
step, then every state field at 1024 fixed cells, full-field L2 norms, totals
and diagnostics).  Here the same rounded initial state is recomputed with the
oracle, loaded into FP64 and mixed-precision contexts in the benchmark's
launch configuration (autotuned tiles, CUDA-graph step), and one step of each
is compared: FP64 within 1e-11 (relative L2 over the sampled cells and in
every full-field norm) with the oracle's Krylov iteration counts; mixed
precision within 1e-5, with Jacobi-PCG and with the Neumann-polynomial CG
(the benchmark's solver).
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hit256_step.json")


@pytest.fixture(scope="module")
def fe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1404_0959_gb300 import build
    build.build()
    from paper_1404_0959_gb300 import fe as fe_mod
    return fe_mod


@pytest.fixture(scope="module")
def case():
    from oracle import piso

    from .golden import make_golden_hit256 as g
    with open(FIXTURE) as f:
        want = json.load(f)
    st = g.rounded_initial_state(piso.Params(**g.PARAMS))
    return g, st, want


def _gpu_step(fe, g, st, precision, solver=None):
    P = g.PARAMS
    s = fe.Solver([dict(N=P["N"], nu=P["nu"], tau_p=P["tau_p"], Y0=P["Y0"], mach_rms=P["mach_rms"],
                        k0=P["k0"], seed=P["seed"])], precision=precision, p_tol=P["p_tol"],
                  p_maxit=P["p_maxit"], solver=fe.FE_PCG_JACOBI if solver is None else solver)
    s.autotune(2)
    s.load_state(0, st)
    s.use_graphs(True)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    out = s.get_state(0)
    d = s.diagnostics(0)
    s.close()
    return out, info[0], d


def _compare(g, out, want, tol):
    f = g.fields({k: out[k] for k in ("rho", "p", "u", "phi", "Y")})
    idx = tuple(np.array(want["cells_zyx"]).T)
    errs = {}
    for k, a in f.items():
        a = np.asarray(a, dtype=np.float64)
        w = np.array(want["samples"][k])
        errs[k] = float(np.linalg.norm(a[idx] - w) / np.linalg.norm(w))
        errs["l2_" + k] = abs(float(np.linalg.norm(a)) / want["l2"][k] - 1)
    assert max(errs.values()) < tol, errs
    return errs


def test_fp64_full_size_matches_oracle(fe, case):
    g, st, want = case
    out, info, d = _gpu_step(fe, g, st, fe.FE_FP64)
    assert info["iters"] == want["iters"]
    assert abs(info["dt"] / want["dt"] - 1) < 1e-14
    _compare(g, out, want, 1e-11)
    assert abs(d["mass"] / want["totals"]["mass"] - 1) < 1e-12
    assert abs(d["dust_mass"][0] / want["totals"]["dust"][0] - 1) < 1e-12
    for k in ("ke", "enstrophy", "taylor", "rho_rms"):
        assert abs(d[k] / want["diag"][k] - 1) < 1e-10, k


@pytest.mark.parametrize("solver", ["jacobi", "poly"])
def test_mixed_full_size_matches_oracle(fe, case, solver):
    g, st, want = case
    out, info, d = _gpu_step(fe, g, st, fe.FE_FP32_MIXED,
                             fe.FE_PCG_POLY if solver == "poly" else fe.FE_PCG_JACOBI)
    assert max(info["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert abs(info["dt"] / want["dt"] - 1) < 1e-6
    _compare(g, out, want, 1e-5)
    assert abs(d["mass"] / want["totals"]["mass"] - 1) < 1e-6
    assert abs(d["dust_mass"][0] / want["totals"]["dust"][0] - 1) < 1e-6
    for k in ("ke", "enstrophy"):
        assert abs(d[k] / want["diag"][k] - 1) < 1e-5, k
