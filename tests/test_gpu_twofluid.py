"""Eulerian two-fluid dust phase on the GPU (dust_model = FE_DUST_TWO_FLUID)
against the oracle (oracle/twofluid.py; the paper's Sec. 2 par. 2 contrasts
the Equilibrium-Eulerian model with this full two-phase model).

Bars: FP64 steps within 1e-11 (relative L2, every field including the dust
velocities) of the oracle step on a ragged grid (N = 24), with three classes,
with the Fourier closure, and over three steps; mixed precision within 1e-5
of the oracle from the same FP32 state; CUDA-graph steps bit-identical to
host-driven steps; every box of an ensemble bit-identical to its solo run;
dust mass conserved to 1e-13 (FP64).
"""
import numpy as np
import pytest

from oracle import piso
from paper_1404_0959_gb300.inputs import random_fields

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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def errors(got, ref):
    e = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"])}
    for d in range(3):
        e["u%d" % d] = rel(got["u"][d], ref["u"][d])
        e["phi%d" % d] = rel(got["phi"][d], ref["phi"][d])
    for j in range(len(ref["Y"])):
        e["Y%d" % j] = rel(got["Y"][j], ref["Y"][j])
        for m in range(3):
            e["V%d%d" % (j, m)] = rel(got["V"][j][m], ref["V"][j][m])
    if ref.get("T") is not None:
        e["T"] = rel(got["T"], ref["T"])
    return e


def case(N, tau, closure=piso.BAROTROPIC, seed=3, slip=True, rounded=False):
    fourier = closure == piso.FOURIER
    rho, u, Y, T = random_fields(N, len(tau), fourier, seed=seed, mach=0.3, noise=0.01)
    if rounded:
        rho, u, Y = f32(rho), [f32(c) for c in u], [f32(y) for y in Y]
        T = f32(T) if fourier else None
    prm = piso.Params(N=N, closure=closure, nu=0.005, tau_p=list(tau), Y0=[0.01] * len(tau),
                      dust_model=piso.TWO_FLUID, p_tol=1e-8 if rounded else 1e-10)
    st = piso.make_state(prm, rho, u, Y, T)
    if slip:  # dust started at the equilibrium particle velocity u - tau Du/Dt
        a = piso.accel(prm, st["rho"], st["u"], st["p"])
        st["V"] = [[st["u"][m] - t * a[m] for m in range(3)] for t in tau]
    if rounded:
        st = {k: ([f32(c) for c in v] if k in ("u", "phi", "Y") else
                  ([[f32(c) for c in vj] for vj in v] if k == "V" else
                   (f32(v) if isinstance(v, np.ndarray) else v))) for k, v in st.items()}
    return prm, st


def solver(fe, prm, precision, **kw):
    return fe.Solver([dict(N=prm.N, nu=prm.nu, tau_p=list(prm.tau_p), Y0=list(prm.Y0))], precision=precision,
                     closure=prm.closure, p_tol=prm.p_tol, dust_model=fe.FE_DUST_TWO_FLUID, **kw)


@pytest.mark.parametrize("N,tau,closure,slip", [(16, (0.05,), piso.BAROTROPIC, True),
                                                (24, (0.02, 0.1, 0.3), piso.BAROTROPIC, True),
                                                (16, (0.02, 0.1, 0.3), piso.FOURIER, True),
                                                (20, (0.1,), piso.BAROTROPIC, False),
                                                (21, (0.05, 0.2), piso.BAROTROPIC, True)])
def test_fp64_two_fluid_step_matches_oracle(fe, N, tau, closure, slip):
    """Even N runs the ring kernels (one class per launch), N = 21 the general column kernels."""
    prm, st = case(N, tau, closure, slip=slip)
    ref, rinfo = piso.step(prm, st)
    s = solver(fe, prm, fe.FE_FP64)
    s.load_state(0, st)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    e = errors(s.get_state(0), ref)
    s.close()
    assert info[0]["iters"] == rinfo["iters"]
    assert max(e.values()) < 1e-11, e


def test_fp64_two_fluid_three_steps_and_conservation(fe):
    prm, st = case(16, (0.02, 0.3), seed=8)
    s = solver(fe, prm, fe.FE_FP64)
    s.load_state(0, st)
    m0 = s.diagnostics(0)["dust_mass"]
    for _ in range(3):
        st, _ = piso.step(prm, st)
        code, _ = s.step(1)
        assert code == fe.FE_OK
    e = errors(s.get_state(0), st)
    m1 = s.diagnostics(0)["dust_mass"]
    s.close()
    assert max(e.values()) < 1e-11, e
    for a, b in zip(m0, m1):
        assert abs(b - a) <= 1e-13 * a


@pytest.mark.parametrize("N", [24, 30])
def test_mixed_two_fluid_step_matches_oracle(fe, N):
    """N = 24 runs the ring kernels, N = 30 (not a multiple of four cells) the general ones."""
    prm, st = case(N, (0.02, 0.1, 0.3), seed=5, rounded=True)
    ref, _ = piso.step(prm, st)
    s = solver(fe, prm, fe.FE_FP32_MIXED)
    s.load_state(0, st)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    e = errors(s.get_state(0), ref)
    s.close()
    assert max(info[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert max(e.values()) < 1e-5, e


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_fluid_graph_steps_equal_host_steps(fe, precision):
    prec = fe.FE_FP64 if precision == "fp64" else fe.FE_FP32_MIXED
    prm, st = case(16, (0.05, 0.2), seed=9, rounded=prec == fe.FE_FP32_MIXED)
    out = []
    for graphs in (False, True):
        s = solver(fe, prm, prec)
        s.load_state(0, st)
        s.use_graphs(graphs)
        code, _ = s.step(3)
        assert code == fe.FE_OK
        out.append(s.get_state(0))
        s.close()
    for j in range(2):
        assert np.array_equal(out[0]["Y"][j], out[1]["Y"][j])
        for m in range(3):
            assert np.array_equal(out[0]["V"][j][m], out[1]["V"][j][m])


def test_two_fluid_ensemble_boxes_equal_solo_runs(fe):
    boxes = [dict(N=16, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=1), dict(N=24, nu=0.004, tau_p=[0.2], Y0=[0.01], seed=2)]
    ens = fe.Solver(boxes, dust_model=fe.FE_DUST_TWO_FLUID)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    code, _ = ens.step(2)
    assert code == fe.FE_OK
    for b, box in enumerate(boxes):
        solo = fe.Solver([box], dust_model=fe.FE_DUST_TWO_FLUID)
        solo.init_state(0, fe.FE_INIT_SPECTRAL)
        code, _ = solo.step(2)
        assert code == fe.FE_OK
        a, c = ens.get_state(b), solo.get_state(0)
        assert np.array_equal(a["Y"][0], c["Y"][0])
        for m in range(3):
            assert np.array_equal(a["V"][0][m], c["V"][0][m])
        solo.close()
    ens.close()


def test_spectral_start_gives_dust_the_gas_velocity(fe):
    s = fe.Solver([dict(N=16, nu=0.005, tau_p=[0.05, 0.1], Y0=[0.01, 0.02], seed=4)], dust_model=fe.FE_DUST_TWO_FLUID)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    st = s.get_state(0)
    for j in range(2):
        for m in range(3):
            assert np.array_equal(st["V"][j][m], st["u"][m])
    s.close()
