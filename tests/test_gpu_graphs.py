"""The CUDA-graph step (Krylov and refinement loops as conditional WHILE
nodes) gives exactly the host-driven step's results: same kernels, same
order, so the comparison is bitwise."""
import numpy as np
import pytest

from paper_1404_0959_gb300.inputs import ensemble64_boxes, random_fields

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


def run(fe, boxes, graphs, nsteps=3, **kw):
    s = fe.Solver(boxes, **kw)
    s.init_state(-1, fe.FE_INIT_SPECTRAL)
    s.use_graphs(graphs)
    code, info = s.step(nsteps)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    out = [s.get_state(b) for b in range(len(boxes))]
    s.close()
    return out, info


def same(a, b):
    for sa, sb in zip(a, b):
        assert np.array_equal(sa["rho"], sb["rho"])
        assert np.array_equal(sa["p"], sb["p"])
        for d in range(3):
            assert np.array_equal(sa["u"][d], sb["u"][d])
            assert np.array_equal(sa["phi"][d], sb["phi"][d])
        for y1, y2 in zip(sa["Y"], sb["Y"]):
            assert np.array_equal(y1, y2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_step_equals_host_step(fe, precision):
    prec = fe.FE_FP64 if precision == "fp64" else fe.FE_FP32_MIXED
    box = [dict(N=32, nu=0.005, tau_p=[0.05], Y0=[0.01], mach_rms=0.3, k0=4.0, seed=3)]
    a, ia = run(fe, box, False, precision=prec, p_tol=1e-8)
    b, ib = run(fe, box, True, precision=prec, p_tol=1e-8)
    same(a, b)
    assert ia[0]["iters"] == ib[0]["iters"]


def test_graph_ensemble_and_bicgstab(fe):
    boxes = ensemble64_boxes(6)
    for b, N in zip(boxes, (16, 24, 32, 48, 16, 24)):
        b["N"] = N
    a, _ = run(fe, boxes, False, precision=fe.FE_FP32_MIXED, p_tol=1e-8)
    b, _ = run(fe, boxes, True, precision=fe.FE_FP32_MIXED, p_tol=1e-8)
    same(a, b)
    box = [dict(N=16, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=1)]
    a, _ = run(fe, box, False, solver=fe.FE_BICGSTAB_JACOBI, transonic=True, p_tol=1e-10)
    b, _ = run(fe, box, True, solver=fe.FE_BICGSTAB_JACOBI, transonic=True, p_tol=1e-10)
    same(a, b)


def test_graph_learned_first_direction(fe):
    from paper_1404_0959_gb300 import learned
    box = [dict(N=32, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=2)]
    res = []
    for graphs in (False, True):
        s = fe.Solver(box, solver=fe.FE_FCG_LEARNED, p_tol=1e-8, learned_every=0)
        s.init_state(0, fe.FE_INIT_SPECTRAL)
        fe.fe_load_preconditioner(s.ctx, learned.he_init(5, zero_last=False))
        s.use_graphs(graphs)
        code, info = s.step(2)
        assert code == fe.FE_OK
        res.append(s.get_state(0))
        s.close()
    same([res[0]], [res[1]])
