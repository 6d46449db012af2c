"""Learned preconditioner against the oracle at the sizes where its
tensor-memory (tcgen05) kernels run.

The stride-1 layers whose output grid is a multiple of 128 cells run on the
fifth-generation tensor cores; the others on warp-level MMA.  Here, at 128^3
(e1a, e1b, u1, out on tcgen05) and 256^3 (also e2 and u2), every layer is
compared with the oracle's convolution (oracle/unet.py, a plain sum over the
27 taps) evaluated in FP64 at a few thousand sampled output voxels, with the
GPU's own stored BF16 input activations, BF16-rounded weights, and the BF16
rounding of the result where the GPU stores BF16.  Bars: relative L2 over the
samples <= 1e-2 per layer and every hidden value within one BF16 rounding of
the oracle's; the FP32 network output (no BF16 storage) within 1e-4.

Then whole PISO steps with the learned pressure solve (flexible CG, Sec. 2
par. 1 pressure-correction equation) after training on the run's own pairs:
mixed precision within 1e-5 of the FP64 oracle step from the same FP32 state
at 32^3 and 128^3, and at 256^3 in the benchmark's launch configuration
(autotuned tiles, CUDA graph) against the stored oracle step
tests/golden/hit256_step.json; every pressure residual <= 1e-8.
"""
import json
import os

import numpy as np
import pytest

from oracle import piso
from oracle import unet as ounet
from paper_1404_0959_gb300.inputs import random_fields, smooth_field

pytestmark = pytest.mark.gpu

NAMES = ["e1a", "e1b", "d1", "e2", "d2", "e3", "u2", "u1", "out"]
LEVEL_CH = [(0, 16), (0, 16), (1, 32), (1, 32), (2, 64), (2, 64), (1, 32), (0, 16)]
# per layer: sources as (activation id, gather mode, channels); 9 = packed network input
SOURCES = {"e1a": [(9, "same", 2)], "e1b": [(0, "same", 16)], "d1": [(1, "down", 16)], "e2": [(2, "same", 32)],
           "d2": [(3, "down", 32)], "e3": [(4, "same", 64)], "u2": [(5, "up", 64), (3, "same", 32)],
           "u1": [(6, "up", 32), (1, "same", 16)], "out": [(7, "same", 16)]}
OUT_LEVEL = {"e1a": 0, "e1b": 0, "d1": 1, "e2": 1, "d2": 2, "e3": 2, "u2": 1, "u1": 0, "out": 0}
FIXTURE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hit256_step.json")
BF16_ULP = 2.0 ** -7
DT = 0.02


@pytest.fixture(scope="module")
def fe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1404_0959_gb300 import build
    build.build()
    from paper_1404_0959_gb300 import fe as fe_mod
    return fe_mod


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = a32.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def flat(P):
    return np.concatenate([np.concatenate([P[n + ".W"].reshape(-1), P[n + ".b"]]) for n in NAMES]).astype(np.float32)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def gather(act, mode, vox, No):
    """Input vectors of the 27 taps at output voxels vox (M, 3) [z, y, x]:
    (M, 27, C).  act: channels-last (n, n, n, C) on the source grid."""
    n = act.shape[0]
    out = np.empty((vox.shape[0], 27, act.shape[3]))
    for ti, t in enumerate(ounet.TAPS):
        t = np.array(t)
        if mode == "same":
            w = (vox + t) % n
        elif mode == "up":  # nearest-neighbour upsampling: fine cell w reads coarse cell w // 2
            w = ((vox + t) % No) // 2
        else:  # stride 2: output v reads input cell 2 v + t
            w = (2 * vox + t) % n
        out[:, ti, :] = act[w[:, 0], w[:, 1], w[:, 2], :]
    return out


def oracle_layer(name, P, acts, vox, No):
    """The oracle's convolution of layer `name` at the sampled voxels, from the
    GPU's stored input activations, with BF16 weights; FP64 sums."""
    xs = [gather(acts[a][..., :C], mode, vox, No) for a, mode, C in SOURCES[name]]
    X = np.concatenate(xs, axis=2)
    W = bf16(P[name + ".W"])
    return np.einsum("mtc,tco->mo", X, W) + P[name + ".b"][None, :]


def network_run(fe, N, seed, want):
    """He-style random network on a random residual; GPU activations of the layers in `want`."""
    import torch
    rho, u, Y, T = random_fields(N, 1, False, seed=seed, noise=0.0)
    s = fe.Solver([dict(N=N, nu=0.002, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED,
                  solver=fe.FE_FCG_LEARNED, p_tol=1e-8)
    s.set_state(0, rho, u, Y)
    P = ounet.init_params(2, seed=seed + 100)
    P["out.W"] *= 0.1  # a correction smaller than the Jacobi direction, as after training
    fe.fe_load_preconditioner(s.ctx, flat(P))
    r = smooth_field(N, seed + 7, 1.0) + 0.1 * np.random.default_rng(seed).standard_normal((N, N, N))
    rt = torch.tensor(r, dtype=torch.float32, device="cuda")
    z = torch.empty_like(rt)
    fe.fe_precond_apply(s.ctx, 0, rt.data_ptr(), DT, z.data_ptr())
    acts = {8: fe.fe_precond_activation(s.ctx, 8, N ** 3).reshape(N, N, N).astype(np.float64)}
    for l in sorted(want):
        if l == 9:
            acts[9] = fe.fe_precond_activation(s.ctx, 9, N ** 3 * 16).reshape(N, N, N, 16).astype(np.float64)
        else:
            lev, C = LEVEL_CH[l]
            n = N >> lev
            acts[l] = fe.fe_precond_activation(s.ctx, l, n ** 3 * C).reshape(n, n, n, C).astype(np.float64)
    out = z.cpu().numpy().astype(np.float64)
    psi = (s.get_field(0, fe.FE_RHO).astype(np.float64) / (1.4 * s.get_field(0, fe.FE_P).astype(np.float64)))
    s.close()
    return P, acts, out, r, psi


def check_layer(name, P, acts, out, N, nsample, rng):
    No = N >> OUT_LEVEL[name]
    vox = rng.integers(0, No, size=(nsample, 3))
    # the grid's wrap-around corners are always among the samples
    vox[:4] = [[0, 0, 0], [No - 1, No - 1, No - 1], [0, No - 1, 0], [No - 1, 0, No - 1]]
    y = oracle_layer(name, P, acts, vox, No)
    if name == "out":
        g = acts[8][vox[:, 0], vox[:, 1], vox[:, 2]]
        e = y[:, 0]
        err = rel(g, e)
        assert err < 1e-4, (name, err)
        return err
    e = bf16(np.maximum(y, 0.0))
    l = NAMES.index(name)
    g = acts[l][vox[:, 0], vox[:, 1], vox[:, 2], :]
    err = rel(g, e)
    scale = np.max(np.abs(e))
    over = np.abs(g - e) > BF16_ULP * np.abs(e) + 1e-6 * scale
    assert err < 1e-2, (name, err)
    assert not over.any(), (name, int(over.sum()), float(np.max(np.abs(g - e))))
    return err


def test_every_layer_at_128_matches_the_oracle_convolution(fe):
    N = 128
    P, acts, out, r, psi = network_run(fe, N, 3, set(range(8)) | {9})
    # the packed input (BF16) and the direction r/d + rms(r) d0 y against the oracle's definitions
    h = 2 * np.pi / N
    x = ounet.network_input(f32(r), psi, DT, h)
    assert rel(acts[9][..., 0], bf16(x[0])) < 1e-2
    assert rel(acts[9][..., 1], bf16(x[1])) < 1e-2
    rho, d0 = ounet.precond_scales(f32(r), DT, h)
    z = f32(r) / ounet.jacobi_diag(psi, DT, h) + rho * d0 * acts[8]
    assert rel(out, z) < 1e-5
    rng = np.random.default_rng(128)
    errs = {name: check_layer(name, P, acts, out, N, 4096, rng) for name in NAMES}
    print("N=128 relative L2 vs the oracle convolution per layer:", {k: "%.2e" % v for k, v in errs.items()})


def test_half_grid_tensor_memory_layers_at_256_match_the_oracle_convolution(fe):
    """At 256^3 the half-grid layers e2 (from d1) and u2 (from up2(e3) and e2)
    also have 128-cell output grids and run on tcgen05."""
    N = 256
    P, acts, out, r, psi = network_run(fe, N, 5, {2, 3, 4, 5, 6})
    rng = np.random.default_rng(256)
    errs = {name: check_layer(name, P, acts, out, N, 4096, rng) for name in ("e2", "u2", "e3")}
    print("N=256 relative L2 vs the oracle convolution:", {k: "%.2e" % v for k, v in errs.items()})


def trained_learned_solver(fe, box, st, precision, learned_every, train_iters=40, tol=1e-8):
    """A learned-solver context whose network was trained on pairs harvested from
    this state's own steps, then reloaded with the state."""
    from paper_1404_0959_gb300 import learned
    s = fe.Solver([box], precision=precision, solver=fe.FE_FCG_LEARNED, p_tol=tol, p_maxit=1000,
                  learned_every=learned_every)
    s.load_state(0, st)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(0))
    bank = learned.PairBank(s, 8)
    bank.harvest(s, 1)
    learned.train(s, bank, train_iters, lr=1e-3)
    s.load_state(0, st)
    return s


def state_errors(got, ref):
    e = {"rho": rel(got["rho"], ref["rho"]), "p": rel(got["p"], ref["p"])}
    for d in range(3):
        e["u%d" % d] = rel(got["u"][d], ref["u"][d])
        e["phi%d" % d] = rel(got["phi"][d], ref["phi"][d])
    for j in range(len(ref["Y"])):
        e["Y%d" % j] = rel(got["Y"][j], ref["Y"][j])
    return e


@pytest.mark.parametrize("N,every", [(32, 0), (32, 1), (128, 0)])
def test_learned_mixed_step_matches_oracle(fe, N, every):
    rho, u, Y, T = random_fields(N, 1, False, seed=9, mach=0.3, noise=0.01)
    prm = piso.Params(N=N, nu=0.002, tau_p=[0.05], Y0=[0.01], p_tol=1e-8)
    st = piso.make_state(prm, f32(rho), [f32(c) for c in u], [f32(y) for y in Y])
    st = {k: ([f32(c) for c in v] if isinstance(v, list) else (f32(v) if isinstance(v, np.ndarray) else v))
          for k, v in st.items()}
    ref, rinfo = piso.step(prm, st)
    box = dict(N=N, nu=0.002, tau_p=[0.05], Y0=[0.01])
    s = trained_learned_solver(fe, box, st, fe.FE_FP32_MIXED, every)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    got = s.get_state(0)
    s.close()
    errs = state_errors(got, ref)
    print("N=%d learned_every=%d iterations %s (oracle PCG %s), max error %.2e"
          % (N, every, info[0]["iters"], rinfo["iters"], max(errs.values())))
    assert max(info[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert max(errs.values()) < 1e-5, errs


def test_learned_full_size_step_matches_stored_oracle_step(fe):
    from .golden import make_golden_hit256 as g
    with open(FIXTURE) as f:
        want = json.load(f)
    P = g.PARAMS
    st = g.rounded_initial_state(piso.Params(**P))
    box = dict(N=P["N"], nu=P["nu"], tau_p=P["tau_p"], Y0=P["Y0"], mach_rms=P["mach_rms"], k0=P["k0"],
               seed=P["seed"])
    s = trained_learned_solver(fe, box, st, fe.FE_FP32_MIXED, 0, train_iters=20)
    s.autotune(1)
    s.load_state(0, st)
    s.use_graphs(True)
    code, info = s.step(1)
    assert code == fe.FE_OK, fe.fe_strerror(code)
    out = s.get_state(0)
    d = s.diagnostics(0)
    s.close()
    assert max(info[0]["rel_res"]) <= 1e-8 * (1 + 1e-3)
    assert abs(info[0]["dt"] / want["dt"] - 1) < 1e-6
    f = g.fields({k: out[k] for k in ("rho", "p", "u", "phi", "Y")})
    idx = tuple(np.array(want["cells_zyx"]).T)
    errs = {}
    for k, a in f.items():
        a = np.asarray(a, dtype=np.float64)
        w = np.array(want["samples"][k])
        errs[k] = float(np.linalg.norm(a[idx] - w) / np.linalg.norm(w))
        errs["l2_" + k] = abs(float(np.linalg.norm(a)) / want["l2"][k] - 1)
    print("256^3 learned step: iterations", info[0]["iters"], "max error %.2e" % max(errs.values()))
    assert max(errs.values()) < 1e-5, errs
    assert abs(d["mass"] / want["totals"]["mass"] - 1) < 1e-6
    for k in ("ke", "enstrophy"):
        assert abs(d[k] / want["diag"][k] - 1) < 1e-5, k
