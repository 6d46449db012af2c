"""CG with the first-order Neumann polynomial preconditioner (solver
FE_PCG_POLY) in FP32 contexts, on the plane-streamed iteration (every N a
power of two in 64..512) and on the z-marching one (any other N), against the
FP64 oracle (oracle/krylov.py: pcg with neumann1) and against the Jacobi
solver.

The preconditioner changes the Krylov space, not the system: mixed-precision
steps meet the reduced-precision bar (1e-5 relative L2 per field) against
the oracle step, a standalone solve reaches the requested FP64-class
residual, and the inner solves take fewer iterations than Jacobi's.  FP64
contexts run plain Jacobi-PCG, bit for bit.
"""
import numpy as np
import pytest

from oracle import krylov, piso
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


def rel(a, b):
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / (nb if nb > 0 else 1.0)


def fields(st):
    out = {"rho": st["rho"], "p": st["p"]}
    for d in range(3):
        out["u%d" % d] = st["u"][d]
        out["phi%d" % d] = st["phi"][d]
    for j, y in enumerate(st["Y"]):
        out["Y%d" % j] = y
    return out


def worst(got, ref):
    g, r = fields(got), fields(ref)
    return max(rel(g[k], r[k]) for k in r)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def solver(fe, N, solver_id, precision=None, seed=1, p_tol=1e-8, **kw):
    rho, u, Y, _ = random_fields(N, 1, False, seed=seed, mach=0.3, noise=0.02)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])],
                  precision=fe.FE_FP32_MIXED if precision is None else precision, p_tol=p_tol, solver=solver_id,
                  **kw)
    s.set_state(0, rho, u, Y)
    return s, (rho, u, Y)


@pytest.mark.parametrize("N", [64, 128])
def test_poly_mixed_step_matches_oracle_in_fewer_iterations(fe, N):
    s, (rho, u, Y) = solver(fe, N, fe.FE_PCG_POLY)
    assert s.plane_streaming_active()
    code, ginf = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    prm = piso.Params(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01], p_tol=1e-10)
    ref, _ = piso.step(prm, piso.make_state(prm, rho, u, Y))
    assert worst(got, ref) <= 1e-5
    j, _ = solver(fe, N, fe.FE_PCG_JACOBI)
    code, jinf = j.step(1)
    assert code == fe.FE_OK
    j.close()
    assert max(ginf[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert sum(ginf[0]["iters"]) < sum(jinf[0]["iters"]), (ginf[0]["iters"], jinf[0]["iters"])


@pytest.mark.parametrize("N", [64, 48, 16])
def test_poly_solve_reaches_fp64_residual_and_oracle_solution(fe, N):
    """64: plane-streamed iteration; 48 and 16: z-marching iteration."""
    import torch
    rho, u, Y, _ = random_fields(N, 1, False, seed=4, noise=0.02)
    prm0 = piso.Params(N=N)
    st = piso.make_state(prm0, f32(rho), [f32(c) for c in u], [f32(Y[0])])
    st = {k: ([f32(c) for c in v] if isinstance(v, list) else (f32(v) if isinstance(v, np.ndarray) else v))
          for k, v in st.items()}
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED,
                  solver=fe.FE_PCG_POLY)
    s.load_state(0, st)
    assert s.plane_streaming_active() == (N == 64)
    psi = f32(np.float32(st["rho"]) / (np.float32(1.4) * np.float32(st["p"])))
    dt = 0.08
    b = f32(random_vector(N, 5))
    matvec, dg = piso.helmholtz(prm0, psi, dt)
    xr, _, _, _ = krylov.pcg(matvec, b, dg, 1e-13, 500, precond=krylov.neumann1(matvec, dg))
    for tol in (1e-8, 1e-10):
        code, x, info = s.solve_pressure(0, torch.tensor(b, dtype=torch.float32, device="cuda"), dt, tol, 500)
        assert code == fe.FE_OK
        assert info.rel_res_true <= tol
        assert rel(x.cpu().numpy(), xr) < 1e-6
    s.close()


def test_poly_solve_256_streamed_blocks_match_oracle(fe):
    """N = 256: the streamed polynomial iteration in its 4096-cell blocks (16 rows of a plane per
    block, four rows of four cells per thread), standalone, against the oracle's Neumann-preconditioned
    PCG solution; then the same solve on the z-marching iteration."""
    import torch
    N = 256
    rho = f32(1.0 + 0.02 * random_vector(N, 11))
    prm0 = piso.Params(N=N)
    st = piso.make_state(prm0, rho, [np.zeros((N, N, N))] * 3, [np.full((N, N, N), 0.01)])
    st = {k: ([f32(c) for c in v] if isinstance(v, list) else (f32(v) if isinstance(v, np.ndarray) else v))
          for k, v in st.items()}
    psi = f32(np.float32(st["rho"]) / (np.float32(1.4) * np.float32(st["p"])))
    dt = 0.02
    b = f32(random_vector(N, 5))
    matvec, dg = piso.helmholtz(prm0, psi, dt)
    xr, _, _, _ = krylov.pcg(matvec, b, dg, 1e-13, 500, precond=krylov.neumann1(matvec, dg))
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    iters = []
    for streaming in (True, False):
        s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED,
                      solver=fe.FE_PCG_POLY)
        s.load_state(0, st)
        s.use_plane_streaming(streaming)
        assert s.plane_streaming_active() == streaming
        code, x, info = s.solve_pressure(0, bt, dt, 1e-10, 500)
        assert code == fe.FE_OK
        assert info.rel_res_true <= 1e-10
        assert rel(x.cpu().numpy(), xr) < 1e-6
        iters.append(info.iters)
        s.close()
    assert abs(iters[0] - iters[1]) <= 1, iters


def test_poly_graph_steps_equal_host_steps(fe):
    out = []
    for graphs in (False, True):
        s = fe.Solver([dict(N=64, nu=0.005, tau_p=[0.05], Y0=[0.01], mach_rms=0.3, k0=4.0, seed=3)],
                      precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=fe.FE_PCG_POLY)
        s.init_state(0, fe.FE_INIT_SPECTRAL)
        s.use_graphs(graphs)
        code, info = s.step(3)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        out.append((s.get_state(0), info[0]["iters"]))
        s.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    for k, v in fields(a).items():
        assert np.array_equal(v, fields(b)[k]), k


def test_poly_fp64_is_jacobi(fe):
    out = []
    for sid in (fe.FE_PCG_POLY, fe.FE_PCG_JACOBI):
        s, _ = solver(fe, 64, sid, precision=fe.FE_FP64, seed=6)
        code, info = s.step(2)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        out.append((s.get_state(0), info[0]["iters"]))
        s.close()
    (a, ia), (b, ib) = out
    assert ia == ib
    for k, v in fields(a).items():
        assert np.array_equal(v, fields(b)[k]), k


# N = 48: rings, z-marching CG; N = 30: not a multiple of four cells, z-marching kernels everywhere
@pytest.mark.parametrize("N", [48, 30])
def test_poly_zmarched_matches_oracle_in_fewer_iterations(fe, N):
    s, (rho, u, Y) = solver(fe, N, fe.FE_PCG_POLY, seed=6)
    assert not s.plane_streaming_active()
    code, ginf = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    prm = piso.Params(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01], p_tol=1e-10)
    ref, _ = piso.step(prm, piso.make_state(prm, rho, u, Y))
    assert worst(got, ref) <= 1e-5
    assert max(ginf[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    j, _ = solver(fe, N, fe.FE_PCG_JACOBI, seed=6)
    code, jinf = j.step(1)
    assert code == fe.FE_OK
    j.close()
    assert sum(ginf[0]["iters"]) < sum(jinf[0]["iters"]), (ginf[0]["iters"], jinf[0]["iters"])


def test_poly_streamed_matches_zmarched(fe):
    out = []
    for streaming in (True, False):
        s, _ = solver(fe, 64, fe.FE_PCG_POLY, seed=7)
        s.use_plane_streaming(streaming)
        assert s.plane_streaming_active() == streaming
        code, info = s.step(2)
        assert code == fe.FE_OK, fe.fe_strerror(code)
        out.append((s.get_state(0), info[0]["iters"]))
        s.close()
    (a, ia), (b, ib) = out
    assert worst(a, b) <= 1e-5
    assert all(abs(x - y) <= 1 for x, y in zip(ia, ib)), (ia, ib)


def test_poly_uneven_ensemble_matches_single_boxes(fe):
    boxes = [dict(N=32, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=3),
             dict(N=48, nu=0.004, tau_p=[0.2], Y0=[0.01], seed=4, mach_rms=0.5)]
    ens = fe.Solver(boxes, precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=fe.FE_PCG_POLY)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    ens.use_graphs(True)
    code, _ = ens.step(2)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    for b, box in enumerate(boxes):
        one = fe.Solver([box], precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=fe.FE_PCG_POLY)
        one.init_state(0, fe.FE_INIT_SPECTRAL)
        code, _ = one.step(2)
        assert code == fe.FE_OK
        assert worst(ens.get_state(b), one.get_state(0)) <= 1e-5
        one.close()
    ens.close()


def test_poly_ensemble_matches_single_boxes(fe):
    boxes = [dict(N=64, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=3),
             dict(N=128, nu=0.002, tau_p=[0.05], Y0=[0.01], seed=4)]
    ens = fe.Solver(boxes, precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=fe.FE_PCG_POLY)
    ens.init_state(-1, fe.FE_INIT_SPECTRAL)
    assert ens.plane_streaming_active()
    code, _ = ens.step(2)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    for b, box in enumerate(boxes):
        one = fe.Solver([box], precision=fe.FE_FP32_MIXED, p_tol=1e-8, solver=fe.FE_PCG_POLY)
        one.init_state(0, fe.FE_INIT_SPECTRAL)
        code, _ = one.step(2)
        assert code == fe.FE_OK
        assert worst(ens.get_state(b), one.get_state(0)) <= 1e-5
        one.close()
    ens.close()


def test_poly_with_transonic_operator_is_refused(fe):
    with pytest.raises(fe.FeError):
        fe.Solver([dict(N=64, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED,
                  solver=fe.FE_PCG_POLY, transonic=1)


def rounded_state(prm, rho, u, Y, T=None):
    st = piso.make_state(prm, f32(rho), [f32(c) for c in u], [f32(y) for y in Y], None if T is None else f32(T))
    out = dict(st)
    for k in ("rho", "p", "T"):
        if st.get(k) is not None:
            out[k] = f32(st[k])
    for k in ("u", "phi", "Y"):
        out[k] = [f32(c) for c in st[k]]
    if st.get("V") is not None:
        out["V"] = [[f32(c) for c in vj] for vj in st["V"]]
    return out


def test_poly_fourier_three_classes_matches_oracle(fe):
    N, tau = 64, (0.02, 0.1, 0.3)
    rho, u, Y, T = random_fields(N, 3, True, seed=11, mach=0.5, noise=0.02)
    prm = piso.Params(N=N, closure=piso.FOURIER, nu=0.002, tau_p=list(tau), Y0=[0.02] * 3, p_tol=1e-8)
    st = rounded_state(prm, rho, u, Y, T)
    ref, _ = piso.step(prm, st)
    s = fe.Solver([dict(N=N, nu=0.002, tau_p=list(tau), Y0=[0.02] * 3)], precision=fe.FE_FP32_MIXED,
                  closure=fe.FE_FOURIER, p_tol=1e-8, solver=fe.FE_PCG_POLY)
    s.load_state(0, st)
    assert s.plane_streaming_active()
    code, ginf = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    assert max(ginf[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert worst(got, ref) <= 1e-5
    assert rel(got["T"], ref["T"]) <= 1e-5


def test_poly_two_fluid_matches_oracle(fe):
    N, tau = 64, (0.05, 0.2)
    rho, u, Y, _ = random_fields(N, 2, False, seed=12, mach=0.3, noise=0.01)
    prm = piso.Params(N=N, nu=0.005, tau_p=list(tau), Y0=[0.01] * 2, dust_model=piso.TWO_FLUID, p_tol=1e-8)
    st = rounded_state(prm, rho, u, Y)
    ref, _ = piso.step(prm, st)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=list(tau), Y0=[0.01] * 2)], precision=fe.FE_FP32_MIXED, p_tol=1e-8,
                  dust_model=fe.FE_DUST_TWO_FLUID, solver=fe.FE_PCG_POLY)
    s.load_state(0, st)
    assert s.plane_streaming_active()
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    assert worst(got, ref) <= 1e-5
    for j in range(2):
        for m in range(3):
            assert rel(got["V"][j][m], ref["V"][j][m]) <= 1e-5, (j, m)


def test_poly_two_way_matches_oracle(fe):
    N, tau = 64, (0.05,)
    rho, u, Y, _ = random_fields(N, 1, False, seed=13, mach=0.3, noise=0.02)
    Y = [20.0 * y for y in Y]  # loading 0.2
    prm = piso.Params(N=N, nu=0.005, tau_p=list(tau), Y0=[0.2], p_tol=1e-8, coupling=piso.TWO_WAY)
    st = rounded_state(prm, rho, u, Y)
    ref, _ = piso.step(prm, st)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=list(tau), Y0=[0.2])], precision=fe.FE_FP32_MIXED, p_tol=1e-8,
                  coupling=fe.FE_COUPLING_TWO_WAY, solver=fe.FE_PCG_POLY)
    s.load_state(0, st)
    assert s.plane_streaming_active()
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    assert worst(got, ref) <= 1e-5
