"""Iso-surfaces and their depth image on the GPU (fe_isosurface,
fe_raster_depth) against the oracle (oracle/isosurface.py; the paper's Fig. 3
shows iso-surfaces of the Q criterion).

The field comes from the seeded input generator, so both sides see the same
numbers: the triangle list (count, order, every coordinate) and the depth
image must be bit for bit the oracle's in FP64 and from FP32 fields (the
extraction is double either way, the image single precision, one rounding
per operation), on grids that
do and do not fill the emit blocks (N = 16, 24, 32); at 128^3 the count and
area, and the triangles of 400 sampled cubes located through the oracle's
per-cube counts.  The Q criterion's iso-surface of a spectral field agrees
with the oracle's from its own Q within 1e-11 (the two Q fields differ by
rounding).  Empty surfaces and a short triangle buffer are handled.
"""
import math

import numpy as np
import pytest

from oracle import diag as odiag
from oracle import isosurface as oiso
from oracle import piso
from paper_1404_0959_gb300.inputs import smooth_field

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


def context(fe, N, precision):
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=precision)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    return s


def gpu_extract(fe, s, field, iso, max_tri):
    import torch
    dt = torch.float64 if s.precision == fe.FE_FP64 else torch.float32
    fd = torch.tensor(field, dtype=dt, device="cuda")
    tri = torch.full((max(max_tri, 1), 9), float("nan"), dtype=torch.float64, device="cuda")
    n, area = fe.fe_isosurface(s.ctx, 0, fd.data_ptr(), iso, tri.data_ptr() if max_tri else None, max_tri)
    return n, area, tri[:min(n, max_tri)], fd


@pytest.mark.parametrize("N", [16, 24, 32])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_triangles_and_depth_bit_for_bit(fe, N, precision):
    import torch
    prec = fe.FE_FP64 if precision == "fp64" else fe.FE_FP32_MIXED
    f = smooth_field(N, 40 + N, 1.0)
    if prec == fe.FE_FP32_MIXED:
        f = f32(f)
    h = 2 * math.pi / N
    T, area = oiso.extract(f, 0.2, h)
    s = context(fe, N, prec)
    n, ga, tri, _ = gpu_extract(fe, s, f, 0.2, len(T) + 5)
    assert n == len(T)
    assert np.array_equal(tri.cpu().numpy().reshape(-1, 3, 3), T)
    assert abs(ga - area) <= 1e-12 * area
    W, L = 3 * N, (N + 1) * h
    depth = torch.empty((W, W), dtype=torch.float32, device="cuda")
    fe.fe_raster_depth(s.ctx, tri.data_ptr(), n, W, L, depth.data_ptr())
    img = oiso.raster_depth(T, W, L)
    assert np.array_equal(depth.cpu().numpy(), img)
    s.close()


def test_large_grid_sampled_cubes(fe):
    N = 128
    f = smooth_field(N, 7, 1.0)
    h = 2 * math.pi / N
    counts = oiso.cube_counts(f, 0.3)
    flat = counts.reshape(-1)
    off = np.concatenate([[0], np.cumsum(flat)])
    s = context(fe, N, fe.FE_FP64)
    n, ga, tri, _ = gpu_extract(fe, s, f, 0.3, int(off[-1]))
    assert n == int(off[-1])
    cut = np.flatnonzero(flat)
    rng = np.random.default_rng(128)
    tri = tri.cpu().numpy().reshape(-1, 3, 3)
    for c in rng.choice(cut, size=400, replace=False):
        k, rem = divmod(int(c), N * N)
        j, i = divmod(rem, N)
        want = np.array(oiso.cube_triangles(f, i, j, k, 0.3, h)).reshape(-1, 3, 3)
        assert np.array_equal(tri[off[c]:off[c + 1]], want), (i, j, k)
    e1 = tri[:, 1] - tri[:, 0]
    e2 = tri[:, 2] - tri[:, 0]
    assert abs(ga - 0.5 * np.sum(np.linalg.norm(np.cross(e1, e2), axis=1))) <= 1e-12 * ga
    s.close()


def test_q_criterion_isosurface_against_the_oracle(fe):
    import torch
    N = 32
    prm = piso.Params(N=N, k0=4.0, mach_rms=0.3, seed=3)
    st = piso.initial_state(prm)
    q = odiag.q_criterion(st["u"], prm.h)
    iso = 0.5 * float(np.std(q))
    T, area = oiso.extract(q, iso, prm.h)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])])
    s.load_state(0, st)
    qd = s.q_criterion(0)
    tri = torch.empty((len(T) + 10, 9), dtype=torch.float64, device="cuda")
    n, ga = fe.fe_isosurface(s.ctx, 0, qd.data_ptr(), iso, tri.data_ptr(), len(T) + 10)
    s.close()
    assert n == len(T)
    assert abs(ga - area) <= 1e-11 * area
    assert np.max(np.abs(tri[:n].cpu().numpy().reshape(-1, 3, 3) - T)) < 1e-11


def test_empty_surface_and_short_buffer(fe):
    import torch
    N = 16
    f = smooth_field(N, 3, 1.0)
    s = context(fe, N, fe.FE_FP64)
    n, a, _, _ = gpu_extract(fe, s, f, 10.0, 0)  # above every value: nothing
    assert n == 0 and a == 0.0
    depth = torch.empty((8, 8), dtype=torch.float32, device="cuda")
    fe.fe_raster_depth(s.ctx, None, 0, 8, 1.0, depth.data_ptr())
    assert torch.isinf(depth).all()
    T, _ = oiso.extract(f, 0.0, 2 * math.pi / N)
    n, a, tri, _ = gpu_extract(fe, s, f, 0.0, 50)
    assert n == len(T) and tri.shape[0] == 50
    assert np.array_equal(tri.cpu().numpy().reshape(-1, 3, 3), T[:50])
    s.close()
