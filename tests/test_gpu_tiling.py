"""Tile depth of the stencil kernels (fe_set_tiling) against the FP64 oracle.

Every z-marching, ring and refinement kernel walks 32 x 8 column tiles tz
planes deep; tz changes which block computes which cell, the ring and queue
prologues at the tile ends, and the order of the partial sums, never the
per-cell arithmetic.  A ragged box (N = 40: neither a multiple of 32 nor of
every tz) is stepped at each depth, including depths beyond N (clamped) and
depths that leave a short last tile, and checked against the oracle at the
FP64 bar (1e-11 relative L2 per field and step) and, in mixed precision, at
the reduced-precision bar (1e-5).
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
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / (nb if nb > 0 else 1.0)


def worst(got, ref):
    pairs = [(got["rho"], ref["rho"]), (got["p"], ref["p"])]
    pairs += [(got["u"][d], ref["u"][d]) for d in range(3)]
    pairs += [(got["phi"][d], ref["phi"][d]) for d in range(3)]
    pairs += [(g, r) for g, r in zip(got["Y"], ref["Y"])]
    return max(rel(g, r) for g, r in pairs)


N = 40


@pytest.fixture(scope="module")
def reference():
    rho, u, Y, _ = random_fields(N, 1, False, seed=7, mach=0.3, noise=0.02)
    prm = piso.Params(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01], p_tol=1e-10)
    ref, info = piso.step(prm, piso.make_state(prm, rho, u, Y))
    return (rho, u, Y), ref


@pytest.mark.parametrize("precision,bar", [(0, 1e-11), (1, 1e-5)])
@pytest.mark.parametrize("tz", [1, 3, 7, 16, 32, 64])
def test_tile_depth_step_matches_oracle(fe, reference, precision, bar, tz):
    (rho, u, Y), ref = reference
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=precision,
                  p_tol=1e-10 if precision == 0 else 1e-8)
    s.set_state(0, rho, u, Y)
    s.set_tiling(tz)
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    assert worst(got, ref) <= bar


def test_per_box_tile_depths_in_an_ensemble(fe):
    """Boxes of one context with different tile depths (fe_set_box_tiling) each match the oracle,
    and the autotuner's per-size pass leaves a tiling under which the step still matches."""
    boxes, refs = [], []
    for n, seed in ((24, 3), (40, 4), (32, 5)):
        rho, u, Y, _ = random_fields(n, 1, False, seed=seed, mach=0.3, noise=0.02)
        prm = piso.Params(N=n, nu=0.005, tau_p=[0.05], Y0=[0.01], p_tol=1e-10)
        ref, _ = piso.step(prm, piso.make_state(prm, rho, u, Y))
        boxes.append((n, rho, u, Y))
        refs.append(ref)
    s = fe.Solver([dict(N=n, nu=0.005, tau_p=[0.05], Y0=[0.01], seed=b + 1) for b, (n, *_r) in enumerate(boxes)],
                  p_tol=1e-10)
    for b, (n, rho, u, Y) in enumerate(boxes):
        s.set_state(b, rho, u, Y)
    for b, tz in enumerate((3, 16, 7)):
        s.set_box_tiling(b, tz)
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    for b in range(3):
        assert worst(s.get_state(b), refs[b]) <= 1e-11
    for b, (n, rho, u, Y) in enumerate(boxes):
        s.set_state(b, rho, u, Y)
    s.autotune(1)
    code, _ = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    for b in range(3):
        assert worst(s.get_state(b), refs[b]) <= 1e-11
    s.close()
