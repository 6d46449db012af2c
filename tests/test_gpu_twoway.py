"""GPU parity of the two-way coupled dusty gas (coupling = FE_COUPLING_TWO_WAY) against the oracle.

The oracle's two-way step (oracle/piso.py) is pinned by tests/test_oracle_twoway.py.  Loadings of
0.1-0.3 per class make the reaction force change the velocity by far more than the bars.  Sizes
cover the ring kernels (N a multiple of the 16-byte chunk) and the z-marching kernels (N = 21 in
FP64, N = 30 in FP32), one class (Ysum read from Y itself) and three classes (Ysum summed by a
kernel); FP64 bar 1e-11, mixed precision 1e-5 per field and step.
"""
import numpy as np
import pytest

from oracle import piso
from paper_1404_0959_gb300.inputs import random_fields

from .test_gpu_mixed import f32, f32_state, state_errors

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


def loaded_fields(N, nd, seed, load=0.2):
    rho, u, Y, _ = random_fields(N, nd, False, seed=seed, mach=0.3, noise=0.02)
    return rho, u, [y * (load / 0.01 / (j + 1)) for j, y in enumerate(Y)]


def pair(fe, N, tau_p, precision, seed=1, coupling=None, p_tol=1e-10):
    coupling = piso.TWO_WAY if coupling is None else coupling
    nd = len(tau_p)
    rho, u, Y = loaded_fields(N, nd, seed)
    prm = piso.Params(N=N, nu=0.005, tau_p=list(tau_p), Y0=[0.2] * nd, p_tol=p_tol, coupling=coupling)
    if precision == "fp64":
        st = piso.make_state(prm, rho, u, Y)
    else:
        st = f32_state(piso.make_state(prm, f32(rho), [f32(c) for c in u], [f32(y) for y in Y]))
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=list(tau_p), Y0=[0.2] * nd)],
                  precision=fe.FE_FP64 if precision == "fp64" else fe.FE_FP32_MIXED, p_tol=p_tol,
                  coupling=fe.FE_COUPLING_TWO_WAY if coupling == piso.TWO_WAY else fe.FE_COUPLING_ONE_WAY)
    s.load_state(0, st)
    return s, prm, st


@pytest.mark.parametrize("N,tau_p", [(24, (0.05,)), (21, (0.05,)), (24, (0.02, 0.1, 0.3)), (21, (0.02, 0.1, 0.3))])
def test_two_way_fp64_matches_oracle(fe, N, tau_p):
    s, prm, st = pair(fe, N, tau_p, "fp64")
    one_way = piso.Params(**{**prm.__dict__, "coupling": piso.ONE_WAY})
    ref = st
    for _ in range(2):
        ref, info = piso.step(prm, ref)
        code, ginf = s.step(1)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        assert abs(ginf[0]["dt"] - info["dt"]) <= 1e-13 * info["dt"]
    e = state_errors(s.get_state(0), ref)
    assert max(e.values()) < 2e-11, e
    # the coupling is not negligible at this loading
    ow = st
    for _ in range(2):
        ow, _ = piso.step(one_way, ow)
    d = state_errors(ow, ref)
    assert d["u0"] > 1e-4 and d["rho"] > 1e-6, d
    s.close()


@pytest.mark.parametrize("N,tau_p", [(32, (0.05,)), (30, (0.05,)), (32, (0.02, 0.1, 0.3))])
def test_two_way_mixed_matches_oracle(fe, N, tau_p):
    s, prm, st = pair(fe, N, tau_p, "mixed", p_tol=1e-8)
    ref, _ = piso.step(prm, st)
    code, ginf = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    assert max(ginf[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    e = state_errors(s.get_state(0), ref)
    assert max(e.values()) < 1e-5, e
    s.close()


def test_two_way_graph_steps_match_host_steps(fe):
    """The CUDA-graph step (captured per state set) and the host-driven step give the same bits."""
    out = []
    for graphs in (True, False):
        s, _prm, _st = pair(fe, 32, (0.02, 0.1), "mixed", p_tol=1e-8)
        s.use_graphs(graphs)
        code, _ = s.step(3)
        assert code == fe.FE_OK
        out.append(s.get_state(0))
        s.close()
    a, b = out
    for k in ("rho", "p"):
        assert np.array_equal(a[k], b[k])
    for m in range(3):
        assert np.array_equal(a["u"][m], b["u"][m])
    for j in range(2):
        assert np.array_equal(a["Y"][j], b["Y"][j])


@pytest.mark.parametrize("closure,model", [(1, 0), (0, 1)])
def test_two_way_scope(fe, closure, model):
    with pytest.raises(fe.FeError) as err:
        fe.Solver([dict(N=16, nu=0.005, tau_p=[0.05], Y0=[0.1])], closure=closure, dust_model=model,
                  coupling=fe.FE_COUPLING_TWO_WAY)
    assert err.value.code == fe.FE_ERR_UNSUPPORTED
