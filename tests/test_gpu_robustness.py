"""Failure handling and solver-pair harvesting through the C ABI.

* A non-finite value in the state (one NaN cell written from the host through
  fe_set_field, a permitted input) must make fe_step return FE_ERR_NONFINITE
  without committing the step: the state stays at level n and the context
  keeps working once a finite state is set again.  FP64 and mixed precision,
  host-driven and CUDA-graph steps.
* A transonic flexible-GMRES context harvests its training pairs with the
  plain BiCGStab of that operator (Sec. 2 par. 1 pressure-correction solve,
  non-symmetric form): every pair (r, e) must satisfy M e = r for the
  operator of one of the step's correctors, which the oracle assembles from
  the same state.
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


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("graphs", [False, True])
def test_nonfinite_state_is_refused_and_not_committed(fe, mixed, graphs):
    N = 16
    rho, u, Y, T = random_fields(N, 1, False, seed=12, noise=0.01)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])],
                  precision=fe.FE_FP32_MIXED if mixed else fe.FE_FP64, p_tol=1e-8, p_maxit=40)
    s.use_graphs(graphs)
    s.set_state(0, rho, u, Y)
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    good = s.get_state(0)
    t_good = s.diagnostics(0)["t"]
    bad_u = np.array(good["u"][0], copy=True)
    bad_u[3, 5, 7] = np.nan
    s.set_field(0, fe.FE_UX, bad_u)
    before = s.get_state(0)
    code, _ = s.step(1)
    assert code == fe.FE_ERR_NONFINITE, fe.fe_strerror(code)
    after = s.get_state(0)
    # not committed: every field is bit for bit the one before the failed step
    for key in ("rho", "p"):
        assert np.array_equal(after[key], before[key], equal_nan=True), key
    for d in range(3):
        assert np.array_equal(after["u"][d], before["u"][d], equal_nan=True)
        assert np.array_equal(after["phi"][d], before["phi"][d], equal_nan=True)
    assert np.array_equal(after["Y"][0], before["Y"][0], equal_nan=True)
    assert s.diagnostics(0)["t"] == t_good
    # the context still works: restore the finite field and step
    s.set_field(0, fe.FE_UX, good["u"][0])
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    st = s.get_state(0)
    assert all(np.isfinite(st[k]).all() for k in ("rho", "p"))
    assert info[0]["rel_res"][0] <= 1e-8 * 1.001
    s.close()


@pytest.mark.parametrize("mixed", [False, True])
def test_harvest_in_transonic_fgmres_context(fe, mixed):
    import torch
    N = 16
    rho, u, Y, T = random_fields(N, 1, False, seed=14, noise=0.01, mach=0.3)
    prm = piso.Params(N=N, transonic=True, p_tol=1e-10)
    st = piso.make_state(prm, rho, u, Y)
    if mixed:
        st = {k: ([f32(c) for c in v] if isinstance(v, list) else (f32(v) if isinstance(v, np.ndarray) else v))
              for k, v in st.items()}
    # the oracle's operators of the step's correctors, recorded while it steps the same state
    ops_seen = []
    orig = piso.helmholtz

    def recording(prm_, psi, dt, HbyA=None):
        mv, dg = orig(prm_, psi, dt, HbyA)
        ops_seen.append(mv)
        return mv, dg

    piso.helmholtz = recording
    try:
        piso.step(prm, st)
    finally:
        piso.helmholtz = orig
    assert len(ops_seen) == 2
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])],
                  precision=fe.FE_FP32_MIXED if mixed else fe.FE_FP64, solver=fe.FE_FGMRES_LEARNED,
                  transonic=True, p_tol=1e-10 if not mixed else 1e-8)
    s.load_state(0, st)
    dtype = torch.float32 if mixed else torch.float64
    b_out = [torch.full((N, N, N), float("nan"), dtype=dtype, device="cuda") for _ in range(8)]
    x_out = [torch.full_like(b_out[0], float("nan")) for _ in range(8)]
    code, got = fe.fe_harvest_pressure(s.ctx, [t.data_ptr() for t in b_out], [t.data_ptr() for t in x_out])
    assert code == fe.FE_OK, fe.fe_strerror(code)
    assert got >= 2
    # residuals are measured against the largest right-hand side of the harvest (the
    # corrector's b): an intermediate pair's e = x* - x_k carries the rounding of x*
    rs = [b_out[k].double().cpu().numpy() for k in range(got)]
    es = [x_out[k].double().cpu().numpy() for k in range(got)]
    rmax = max(np.linalg.norm(r) for r in rs)
    bar = 1e-5 if mixed else 1e-8
    worst = 0.0
    for k, (r, e) in enumerate(zip(rs, es)):
        assert np.isfinite(r).all() and np.isfinite(e).all()
        assert np.linalg.norm(r) > 0 and np.linalg.norm(e) > 0
        err = min(np.linalg.norm(mv(e) - r) for mv in ops_seen) / rmax
        worst = max(worst, err)
        assert err < bar, (k, err)
    print("transonic harvest (%s): %d pairs, worst ||M e - r|| / max ||r|| = %.2e"
          % ("mixed" if mixed else "fp64", got, worst))
    s.close()
