"""The C-ABI library builds, loads and exports every entry point of include/fe.h.

CPU only: no call here touches a GPU (argument validation happens before any
CUDA call, so rejected parameter sets are checked too).
"""
import ctypes
import os
import re

import pytest

from paper_1404_0959_gb300 import build as fe_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fe_build.build()
    from paper_1404_0959_gb300 import fe
    return fe.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "fe.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+\*?(fe_\w+)\s*\(", text, flags=re.M)))


def test_header_parses_and_lists_entry_points():
    names = declared_functions()
    for n in ("fe_create", "fe_init_state", "fe_step", "fe_solve_pressure", "fe_diagnostics", "fe_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_uses_the_c_names():
    from paper_1404_0959_gb300 import fe
    for name in declared_functions():
        assert hasattr(fe, name), name


def test_strerror(lib):
    assert lib.fe_strerror(0) == b"ok"
    assert b"converge" in lib.fe_strerror(-3)
    assert lib.fe_strerror(12345) == b"unknown error"


def _params(**kw):
    from paper_1404_0959_gb300 import fe
    keep = []
    N = (ctypes.c_int32 * 1)(kw.pop("N", 16))
    nu = (ctypes.c_double * 1)(0.005)
    mach = (ctypes.c_double * 1)(0.2)
    k0 = (ctypes.c_double * 1)(4.0)
    seed = (ctypes.c_uint64 * 1)(0)
    tau = (ctypes.c_double * 1)(0.05)
    y0 = (ctypes.c_double * 1)(0.01)
    keep += [N, nu, mach, k0, seed, tau, y0]
    p = fe.fe_params(1, N, 0, 0, 1.4, 0.7, nu, 1, tau, y0, mach, k0, seed, 0.5, 1.2, 0.0, 2, 0, 1e-10, 100, 0, 1)
    for k, v in kw.items():
        setattr(p, k, v)
    return p, keep


@pytest.mark.parametrize("field,value", [("n_boxes", 0), ("precision", 7), ("closure", 3), ("n_dust", 9),
                                         ("n_corr", 0), ("gamma", 1.0), ("cfl", 0.0), ("p_tol", 0.0),
                                         ("p_maxit", 0), ("solver", 9), ("transonic", 1)])
def test_invalid_params_rejected_before_any_cuda_call(lib, field, value):
    from paper_1404_0959_gb300 import fe
    p, keep = _params(**{field: value})
    ctx = ctypes.c_void_p()
    assert lib.fe_create(ctypes.byref(p), None, ctypes.byref(ctx)) == fe.FE_ERR_INVALID_ARG
    assert not ctx.value


@pytest.mark.parametrize("N", [4, 600])
def test_grid_size_limits(lib, N):
    from paper_1404_0959_gb300 import fe
    p, keep = _params(N=N)
    ctx = ctypes.c_void_p()
    assert lib.fe_create(ctypes.byref(p), None, ctypes.byref(ctx)) == fe.FE_ERR_INVALID_ARG


def test_null_arguments(lib):
    from paper_1404_0959_gb300 import fe
    assert lib.fe_create(None, None, None) == fe.FE_ERR_INVALID_ARG
    assert lib.fe_step(None, 1, None) == fe.FE_ERR_INVALID_ARG
    assert lib.fe_init_state(None, 0, 0) == fe.FE_ERR_INVALID_ARG
    lib.fe_destroy(None)


@pytest.mark.parametrize("solver", ["FE_FCG_LEARNED", "FE_FGMRES_LEARNED"])
def test_learned_solvers_need_one_box_with_n_divisible_by_four(lib, solver):
    """The U-Net halves the grid twice, so the learned solvers take one box
    with N % 4 == 0; other grids are refused before any CUDA call."""
    from paper_1404_0959_gb300 import fe
    p, keep = _params(N=18, solver=getattr(fe, solver))
    ctx = ctypes.c_void_p()
    assert lib.fe_create(ctypes.byref(p), None, ctypes.byref(ctx)) == fe.FE_ERR_UNSUPPORTED
    assert not ctx.value


def test_fgmres_accepts_the_transonic_operator_and_fcg_does_not(lib):
    """Flexible CG needs a symmetric operator; flexible GMRES does not.  The
    FCG refusal comes from validation (no CUDA call); the FGMRES parameters
    pass validation, so on a machine without a GPU fe_create fails later, at
    its first CUDA call, with FE_ERR_CUDA rather than a parameter error."""
    import torch
    from paper_1404_0959_gb300 import fe
    p, keep = _params(N=16, solver=fe.FE_FCG_LEARNED, transonic=1)
    ctx = ctypes.c_void_p()
    assert lib.fe_create(ctypes.byref(p), None, ctypes.byref(ctx)) == fe.FE_ERR_UNSUPPORTED
    if torch.cuda.is_available():
        pytest.skip("the no-GPU branch of this check needs a machine without a GPU")
    p, keep = _params(N=16, solver=fe.FE_FGMRES_LEARNED, transonic=1)
    rc = lib.fe_create(ctypes.byref(p), None, ctypes.byref(ctx))
    assert rc not in (fe.FE_ERR_INVALID_ARG, fe.FE_ERR_UNSUPPORTED, fe.FE_OK)
    assert not ctx.value
