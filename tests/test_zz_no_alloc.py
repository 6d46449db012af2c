"""Allocation-free pressure solve against the context-based one.

fe_solve_pressure_noalloc serves callers that cannot allocate device memory
(for instance code running while another framework owns the device
allocator, or loops that must never allocate): it keeps its Krylov vectors
in a fixed static device array instead of a context.  Through the C ABI it
must return the same correction as fe_solve_pressure, call after call, since
the static array is reused and keeps the previous call's contents.
"""
import ctypes

import numpy as np
import pytest

from paper_1404_0959_gb300.inputs import random_fields, random_vector

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


def test_noalloc_solve_matches_context_solve_on_consecutive_calls(fe):
    import torch
    N, dt, tol = 40, 0.09, 1e-10
    rho, u, Y, T = random_fields(N, 1, False, seed=21, noise=0.02)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.set_state(0, rho, u, Y)
    rho_d = s.get_field(0, fe.FE_RHO, device=True)
    p_d = s.get_field(0, fe.FE_P, device=True)
    psi = (rho_d / (1.4 * p_d)).contiguous()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        b = torch.tensor(random_vector(N, 30 + call), device="cuda")
        code_ref, x_ref, info_ref = s.solve_pressure(0, b, dt, tol, 500)
        assert code_ref == fe.FE_OK
        x = torch.full_like(b, float("nan"))
        info = fe.fe_solve_info()
        code = fe.lib().fe_solve_pressure_noalloc(N, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                                  ctypes.c_void_p(x.data_ptr()), dt, tol, 500,
                                                  ctypes.c_void_p(stream), ctypes.byref(info))
        torch.cuda.synchronize()
        assert code == fe.FE_OK, fe.fe_strerror(code)
        assert abs(info.iters - info_ref.iters) <= 1
        assert info.rel_res_true < tol
        xr = x_ref.cpu().numpy()
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err < 1e-10, (call, err)
    s.close()


def test_noalloc_rejects_grids_beyond_its_static_buffer(fe):
    import torch
    N = fe.FE_NOALLOC_MAX_N + 1
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    info = fe.fe_solve_info()
    code = fe.lib().fe_solve_pressure_noalloc(N, ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                                              ctypes.c_void_p(dummy.data_ptr()), 0.1, 1e-8, 10, None,
                                              ctypes.byref(info))
    assert code == fe.FE_ERR_TOO_LARGE
    assert "static buffer" in fe.fe_strerror(code)


def test_noalloc_at_its_maximum_grid_matches_the_oracle_pcg(fe):
    """N = FE_NOALLOC_MAX_N, the largest grid the static array holds, against the
    FP64 oracle's Jacobi-PCG on the same operator (Sec. 2 par. 1 pressure solve),
    twice in a row so the second call starts from the first call's leftovers."""
    import torch
    from oracle import krylov, piso
    from paper_1404_0959_gb300.inputs import smooth_field
    N, dt, tol = fe.FE_NOALLOC_MAX_N, 0.05, 1e-10
    prm = piso.Params(N=N)
    psi_h = 1.0 + smooth_field(N, 41, 0.2)
    psi = torch.tensor(psi_h, device="cuda")
    matvec, dg = piso.helmholtz(prm, psi_h, dt)
    for call in range(2):
        b_h = random_vector(N, 50 + call)
        xr, _, _, _ = krylov.pcg(matvec, b_h, dg, 1e-13, 1000)
        b = torch.tensor(b_h, device="cuda")
        x = torch.full_like(b, float("nan"))
        info = fe.fe_solve_info()
        code = fe.lib().fe_solve_pressure_noalloc(N, ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                                  ctypes.c_void_p(x.data_ptr()), dt, tol, 1000, None,
                                                  ctypes.byref(info))
        torch.cuda.synchronize()
        assert code == fe.FE_OK, fe.fe_strerror(code)
        assert info.rel_res_true < tol
        err = np.linalg.norm(x.cpu().numpy() - xr) / np.linalg.norm(xr)
        assert err < 1e-9, (call, err)


def test_noalloc_refuses_a_capturing_stream(fe):
    """The solve polls its convergence flag from the host, so it cannot be
    recorded into a CUDA graph: on a capturing stream it must refuse before
    enqueueing anything, and the capture must still end cleanly."""
    import torch
    N = 16
    a = torch.ones(N ** 3, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(a)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    info = fe.fe_solve_info()
    with torch.cuda.stream(s):
        g.capture_begin()
        code = fe.lib().fe_solve_pressure_noalloc(N, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                                  ctypes.c_void_p(x.data_ptr()), 0.1, 1e-8, 10,
                                                  ctypes.c_void_p(s.cuda_stream), ctypes.byref(info))
        g.capture_end()
    torch.cuda.synchronize()
    assert code == fe.FE_ERR_UNSUPPORTED
