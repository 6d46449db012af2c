"""Ensembles: independent boxes of uneven N, Mach and Stokes number advanced
by one launch per stage.  Every box must equal the same box run alone
(bitwise: identical tiles, reductions and Krylov iterations), and in FP64
every box must match the oracle to 1e-11."""
import numpy as np
import pytest

from oracle import ic as oic
from oracle import piso
from paper_1404_0959_gb300.inputs import ensemble64_boxes

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


def small_boxes(n=8):
    boxes = ensemble64_boxes(n)
    for b, N in zip(boxes, (16, 24, 32, 48, 16, 24, 32, 48)):
        b["N"] = N
    return boxes


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_each_box_equals_its_solo_run(fe, precision):
    prec = fe.FE_FP32_MIXED if precision == "mixed" else fe.FE_FP64
    boxes = small_boxes()
    ens = fe.Solver(boxes, precision=prec, p_tol=1e-8)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    code, info = ens.step(3)
    assert code == fe.FE_OK
    for i, b in enumerate(boxes):
        solo = fe.Solver([b], precision=prec, p_tol=1e-8)
        solo.init_state(0, fe.FE_INIT_SPECTRAL)
        c2, inf2 = solo.step(3)
        assert c2 == fe.FE_OK
        a = ens.get_state(i)
        s = solo.get_state(0)
        assert np.array_equal(a["rho"], s["rho"]), i
        for d in range(3):
            assert np.array_equal(a["u"][d], s["u"][d]), (i, d)
        assert np.array_equal(a["Y"][0], s["Y"][0]), i
        assert info[i]["iters"] == inf2[0]["iters"]
        assert info[i]["dt"] == inf2[0]["dt"]
        solo.close()
    ens.close()


def test_fp64_ensemble_boxes_match_oracle(fe):
    boxes = small_boxes(4)
    ens = fe.Solver(boxes, precision=fe.FE_FP64, p_tol=1e-10)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    code, _ = ens.step(1)
    assert code == fe.FE_OK
    for i, b in enumerate(boxes):
        prm = piso.Params(N=b["N"], nu=b["nu"], tau_p=b["tau_p"], Y0=b["Y0"], mach_rms=b["mach_rms"], k0=b["k0"],
                          seed=b["seed"], p_tol=1e-10)
        st = piso.initial_state(prm)
        ref, _ = piso.step(prm, st)
        got = ens.get_state(i)
        for k in ("rho", "p"):
            err = np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
            assert err < 1e-11, (i, k, err)
        for d in range(3):
            err = np.linalg.norm(got["u"][d] - ref["u"][d]) / np.linalg.norm(ref["u"][d])
            assert err < 1e-11, (i, d, err)
    ens.close()


def test_ensemble64_workload_runs(fe):
    """The 64-box workload (N in {32,48,64,96}, M in {0.2,0.5}, tau_p in [0.02,0.5])."""
    boxes = ensemble64_boxes(64)
    ens = fe.Solver(boxes, precision=fe.FE_FP32_MIXED, p_tol=1e-8)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    d0 = [ens.diagnostics(i)["mass"] for i in range(64)]
    code, info = ens.step(2)
    assert code == fe.FE_OK
    for i in range(64):
        assert max(info[i]["rel_res"]) <= 1e-8 * (1 + 1e-3)
        m = ens.diagnostics(i)["mass"]
        assert abs(m - d0[i]) <= 1e-6 * d0[i]
    ens.close()
