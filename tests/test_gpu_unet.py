"""Learned preconditioner: GPU U-Net (BF16 tensor cores, FP32 accumulation)
against the FP64 oracle U-Net, training on solver-generated pairs, flexible
CG with the network, and the gain over the method without it.

The network corrects the Jacobi direction (residual form, oracle/unet.py):
input [(r/d) / (rms(r) d0), (3 dt/h^2) / d], direction z = r/d + rms(r) d0 y.

Bars: forward output within 2e-2 (relative L2) of the FP64 oracle; every
layer's weight and bias gradient within 3e-2 of the oracle evaluated with
BF16 rounding at the points where the GPU stores BF16 (random-network
gradients are sums with heavy cancellation, so plain FP64 is no yardstick for
them); flexible CG
reaches the same residual as Jacobi-PCG and falls back to Jacobi directions
when the network gives a non-descent direction.
"""
import time

import numpy as np
import pytest

from oracle import krylov, piso
from oracle import unet as ounet
from paper_1404_0959_gb300.inputs import random_fields, smooth_field

pytestmark = pytest.mark.gpu

NAMES = ["e1a", "e1b", "d1", "e2", "d2", "e3", "u2", "u1", "out"]


@pytest.fixture(scope="module")
def fe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1404_0959_gb300 import build
    build.build()
    from paper_1404_0959_gb300 import fe as fe_mod
    return fe_mod


def flat(P):
    return np.concatenate([np.concatenate([P[n + ".W"].reshape(-1), P[n + ".b"]]) for n in NAMES]).astype(np.float32)


def unflat(w, P):
    out, off = {}, 0
    for n in NAMES:
        sh = P[n + ".W"].shape
        k = int(np.prod(sh))
        out[n + ".W"] = w[off:off + k].reshape(sh).astype(np.float64)
        off += k
        cb = P[n + ".b"].size
        out[n + ".b"] = w[off:off + cb].astype(np.float64)
        off += cb
    return out


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


DT = 0.08


def make(fe, N, solver=None, seed=1):
    rho, u, Y, T = random_fields(N, 1, False, seed=seed, noise=0.0)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])],
                  solver=fe.FE_FCG_LEARNED if solver is None else solver, p_tol=1e-8)
    s.set_state(0, rho, u, Y)
    prm = piso.Params(N=N)
    st = piso.make_state(prm, rho, u, Y)
    psi = st["rho"] / (prm.gamma * st["p"])
    return s, psi


def oracle_input(r, psi, N, dt=DT):
    return ounet.network_input(r, psi, dt, 2 * np.pi / N)


def test_forward_matches_oracle(fe):
    import torch
    N = 16
    s, psi = make(fe, N)
    P = ounet.init_params(2, seed=3)
    fe.fe_load_preconditioner(s.ctx, flat(P))
    r = smooth_field(N, 7, 1.0) + 0.1 * np.random.default_rng(8).standard_normal((N, N, N))
    rt = torch.tensor(r, device="cuda")
    z = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    fe.fe_precond_apply(s.ctx, 0, rt.data_ptr(), DT, z.data_ptr())
    y, _ = ounet.forward(P, oracle_input(r, psi, N))
    yg = fe.fe_precond_activation(s.ctx, 8, N ** 3).reshape(N, N, N)
    assert rel(yg, y[0]) < 2e-2
    # the direction: Jacobi plus the scaled network correction
    assert rel(z.cpu().numpy(), ounet.direction(P, r, psi, DT, 2 * np.pi / N)) < 2e-2
    # the weights read back are the ones loaded
    w = fe.fe_get_preconditioner(s.ctx)
    assert np.array_equal(w, flat(P))
    s.close()


def test_zero_last_layer_is_the_jacobi_direction(fe):
    """The default initial network (output layer zero) gives exactly r / d."""
    import torch
    from paper_1404_0959_gb300 import learned
    N = 16
    s, psi = make(fe, N)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(2))
    r = np.random.default_rng(3).standard_normal((N, N, N))
    rt = torch.tensor(r, device="cuda")
    z = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    fe.fe_precond_apply(s.ctx, 0, rt.data_ptr(), DT, z.data_ptr())
    d = ounet.jacobi_diag(psi, DT, 2 * np.pi / N)
    assert rel(z.cpu().numpy(), r / d) < 1e-6  # FP32 output
    s.close()


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    b = a32.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def quantised_forward_backward(P, x, t):
    """The oracle's layers with BF16 rounding where the GPU path stores BF16:
    weights, network input, every hidden activation, and every layer's
    pre-activation gradient; sums, the output and the data gradients stay wide."""
    Q = {k: (bf16(v) if k.endswith(".W") else v) for k, v in P.items()}
    c = {"x": bf16(x)}
    conv, relu, up2 = ounet.conv, ounet.relu, ounet.up2
    c["e1a"] = bf16(relu(conv(c["x"], Q["e1a.W"], Q["e1a.b"])))
    c["e1b"] = bf16(relu(conv(c["e1a"], Q["e1b.W"], Q["e1b.b"])))
    c["d1"] = bf16(relu(conv(c["e1b"], Q["d1.W"], Q["d1.b"], 2)))
    c["e2"] = bf16(relu(conv(c["d1"], Q["e2.W"], Q["e2.b"])))
    c["d2"] = bf16(relu(conv(c["e2"], Q["d2.W"], Q["d2.b"], 2)))
    c["e3"] = bf16(relu(conv(c["d2"], Q["e3.W"], Q["e3.b"])))
    c["u2in"] = np.concatenate([up2(c["e3"]), c["e2"]], axis=0)
    c["u2"] = bf16(relu(conv(c["u2in"], Q["u2.W"], Q["u2.b"])))
    c["u1in"] = np.concatenate([up2(c["u2"]), c["e1b"]], axis=0)
    c["u1"] = bf16(relu(conv(c["u1in"], Q["u1.W"], Q["u1.b"])))
    y = conv(c["u1"], Q["out.W"], Q["out.b"])
    L, dy = ounet.loss_rel_mse(y, t)
    cb = ounet.conv_backward
    G = {}
    d = bf16(dy)
    d, G["out.W"], G["out.b"] = cb(c["u1"], Q["out.W"], d)
    d = bf16(d * (c["u1"] > 0))
    d, G["u1.W"], G["u1.b"] = cb(c["u1in"], Q["u1.W"], d)
    sk1 = d[32:]
    d = bf16(ounet.up2_backward(d[:32]) * (c["u2"] > 0))
    d, G["u2.W"], G["u2.b"] = cb(c["u2in"], Q["u2.W"], d)
    sk2 = d[64:]
    d = bf16(ounet.up2_backward(d[:64]) * (c["e3"] > 0))
    d, G["e3.W"], G["e3.b"] = cb(c["d2"], Q["e3.W"], d)
    d = bf16(d * (c["d2"] > 0))
    d, G["d2.W"], G["d2.b"] = cb(c["e2"], Q["d2.W"], d, 2)
    d = bf16((d + sk2) * (c["e2"] > 0))
    d, G["e2.W"], G["e2.b"] = cb(c["d1"], Q["e2.W"], d)
    d = bf16(d * (c["d1"] > 0))
    d, G["d1.W"], G["d1.b"] = cb(c["e1b"], Q["d1.W"], d, 2)
    d = bf16((d + sk1) * (c["e1b"] > 0))
    d, G["e1b.W"], G["e1b.b"] = cb(c["e1a"], Q["e1b.W"], d)
    d = bf16(d * (c["e1a"] > 0))
    _, G["e1a.W"], G["e1a.b"] = cb(c["x"], Q["e1a.W"], d)
    return y, L, G


LEVEL_CH = [(0, 16), (0, 16), (1, 32), (1, 32), (2, 64), (2, 64), (1, 32), (0, 16)]


def test_every_layer_matches_quantised_oracle(fe):
    import torch
    N = 16
    s, psi = make(fe, N, seed=2)
    P = ounet.init_params(2, seed=4)
    fe.fe_load_preconditioner(s.ctx, flat(P))
    r = smooth_field(N, 10, 1.0) + 0.1 * np.random.default_rng(9).standard_normal((N, N, N))
    z = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
    rt = torch.tensor(r, device="cuda")
    fe.fe_precond_apply(s.ctx, 0, rt.data_ptr(), DT, z.data_ptr())
    x = oracle_input(r, psi, N)
    xin = fe.fe_precond_activation(s.ctx, 9, N ** 3 * 16).reshape(N, N, N, 16)
    assert rel(xin[..., :2].transpose(3, 0, 1, 2), bf16(x)) < 1e-6
    Q = {k: (bf16(v) if k.endswith(".W") else v) for k, v in P.items()}
    conv, relu, up2 = ounet.conv, ounet.relu, ounet.up2
    acts = {}
    a = bf16(x)
    seq = [("e1a", None, 1), ("e1b", None, 1), ("d1", None, 2), ("e2", None, 1), ("d2", None, 2), ("e3", None, 1)]
    for name, _u, stride in seq:
        a = bf16(relu(conv(a, Q[name + ".W"], Q[name + ".b"], stride)))
        acts[name] = a
    acts["u2"] = bf16(relu(conv(np.concatenate([up2(acts["e3"]), acts["e2"]]), Q["u2.W"], Q["u2.b"])))
    acts["u1"] = bf16(relu(conv(np.concatenate([up2(acts["u2"]), acts["e1b"]]), Q["u1.W"], Q["u1.b"])))
    errs = {}
    for l, name in enumerate(NAMES[:8]):
        lev, C = LEVEL_CH[l]
        n = N >> lev
        g = fe.fe_precond_activation(s.ctx, l, n ** 3 * C).reshape(n, n, n, C).transpose(3, 0, 1, 2)
        # GPU layer input is its own previous layer: compare the layer given the oracle's activations
        errs[name] = rel(g, acts[name])
    print("per-layer relative errors vs the BF16-matched oracle:", {k: round(v, 5) for k, v in errs.items()})
    assert max(errs.values()) < 1e-2, errs
    s.close()


def test_gradients_match_oracle(fe):
    import torch
    N = 16
    s, psi = make(fe, N, seed=2)
    P = ounet.init_params(2, seed=4)
    fe.fe_load_preconditioner(s.ctx, flat(P))
    rng = np.random.default_rng(9)
    r = smooth_field(N, 10, 1.0) + 0.1 * rng.standard_normal((N, N, N))
    # a correction e whose network target (e - r/d) / (rms(r) d0) is a unit-scale smooth field, the
    # scale the residual form trains at
    h = 2 * np.pi / N
    rho_r, d0 = ounet.precond_scales(r, DT, h)
    e = r / ounet.jacobi_diag(psi, DT, h) + rho_r * d0 * smooth_field(N, 11, 1.0)
    rt = torch.tensor(r, device="cuda")  # keep both tensors alive while the library reads them
    et = torch.tensor(e, device="cuda")
    loss = fe.fe_precond_train_step(s.ctx, 0, rt.data_ptr(), et.data_ptr(), DT, 0.0)
    g = unflat(fe.fe_get_preconditioner(s.ctx, gradients=True), P)
    t = ounet.training_target(r, e, psi, DT, 2 * np.pi / N)
    # FP64 oracle: the loss agrees to BF16 level
    y, cache = ounet.forward(P, oracle_input(r, psi, N))
    L, dy = ounet.loss_rel_mse(y, t)
    assert abs(loss - L) < 5e-2 * L
    # with BF16 rounding at the GPU's storage points the gradients agree closely
    yq, Lq, Gq = quantised_forward_backward(P, oracle_input(r, psi, N), t)
    assert abs(loss - Lq) < 2e-3 * Lq
    errs = {n + k: rel(g[n + k], Gq[n + k]) for n in NAMES for k in (".W", ".b")}
    print("relative gradient errors vs the BF16-matched oracle:", {k: round(v, 4) for k, v in errs.items()})
    # BF16 rounding of each layer's pre-activation gradient compounds toward the input layer
    assert max(errs.values()) < 3e-2, errs
    s.close()


def test_training_reduces_loss(fe):
    import torch
    N = 16
    s, psi = make(fe, N, seed=5)
    from paper_1404_0959_gb300 import learned
    fe.fe_load_preconditioner(s.ctx, learned.he_init(0, zero_last=False))
    r = torch.tensor(smooth_field(N, 12, 1.0), device="cuda")
    e = torch.tensor(smooth_field(N, 12, 1.0) * 0.5 + smooth_field(N, 13, 0.2), device="cuda")
    losses = [fe.fe_precond_train_step(s.ctx, 0, r.data_ptr(), e.data_ptr(), DT, 2e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0], (losses[0], losses[-1])
    s.close()


def test_flexible_cg_converges_with_any_network(fe):
    """Random and adversarial (sign-flipped) networks: same solution as PCG."""
    import torch
    from paper_1404_0959_gb300 import learned
    N = 32
    s, psi = make(fe, N, seed=6)
    dt = 0.1
    b = torch.tensor(smooth_field(N, 14, 1.0), device="cuda")
    prm = piso.Params(N=N)
    matvec, dg = piso.helmholtz(prm, psi, dt)
    xr, _, _, _ = krylov.pcg(matvec, b.cpu().numpy(), dg, 1e-13, 500)
    for sign in (1.0, -1.0):
        w = learned.he_init(1, zero_last=False)
        n_out = 27 * 16 * 1 + 1
        w[-n_out:] *= sign
        fe.fe_load_preconditioner(s.ctx, w)
        code, x, info = s.solve_pressure(0, b, dt, 1e-8, 300)
        assert code == fe.FE_OK
        assert info.rel_res_true <= 1e-8
        assert rel(x.cpu().numpy(), xr) < 1e-6
    s.close()


def test_trained_network_gain(fe):
    """What the trained network gains over the method without it.

    64^3 box with the 32^3 workload's physics (spectral decaying turbulence,
    Mach 0.2, k0 4, nu 0.005).  Training pairs are harvested from this run's
    own plain solves over eight steps; the fresh systems come from the step
    after them.  Each is solved to a 1e-8 residual by Jacobi-PCG (the method
    without the network), by flexible CG with the untrained network (output
    layer zero: exactly the Jacobi direction), and by flexible CG with the
    trained network applied every iteration and as the first direction only.
    Every solve must reach the tolerance; the trained network must need fewer
    iterations in total than Jacobi-PCG.
    """
    import torch
    from paper_1404_0959_gb300 import learned
    from paper_1404_0959_gb300.inputs import WORKLOADS
    w = WORKLOADS["hit32"]
    N = 64
    box = dict(N=N, nu=w["nu"], tau_p=w["tau_p"], Y0=w["Y0"], mach_rms=w["mach_rms"], k0=w["k0"], seed=0)
    s = fe.Solver([box], solver=fe.FE_FCG_LEARNED, p_tol=1e-8, learned_every=1)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(0))
    bank = learned.PairBank(s, 48)
    bank.harvest(s, 8)
    test = learned.PairBank(s, 6)
    test.harvest(s, 1)
    plain = fe.Solver([box], solver=fe.FE_PCG_JACOBI, p_tol=1e-8)
    plain.load_state(0, s.get_state(0))
    first = fe.Solver([box], solver=fe.FE_FCG_LEARNED, p_tol=1e-8, learned_every=0)
    first.load_state(0, s.get_state(0))

    def solve_all(ctx_solver):
        out = []
        for k in range(test.n):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c, x, inf = ctx_solver.solve_pressure(0, test.b[k], test.dt[k], 1e-8, 400)
            torch.cuda.synchronize()
            out.append((c, inf.iters, inf.rel_res_true, time.perf_counter() - t0))
        return out

    untrained = solve_all(s)
    t0 = time.perf_counter()
    hist = learned.train(s, bank, 600, lr=1e-3)
    train_s = time.perf_counter() - t0
    trained = solve_all(s)
    fe.fe_load_preconditioner(first.ctx, fe.fe_get_preconditioner(s.ctx))
    once = solve_all(first)
    base = solve_all(plain)
    tot = lambda res: sum(a[1] for a in res)
    print("iterations to 1e-8 per system [Jacobi-PCG, untrained (= Jacobi), trained every iteration, trained first "
          "direction only]:", [(c[1], a[1], b[1], d[1]) for a, b, c, d in zip(untrained, trained, base, once)],
          "totals", (tot(base), tot(untrained), tot(trained), tot(once)),
          "seconds per solve", (round(np.mean([c[3] for c in base]), 4), round(np.mean([b[3] for b in trained]), 4)),
          "loss %.3e -> %.3e in %.1f s" % (hist[0], hist[-1], train_s))
    for res in (untrained, trained, base, once):
        for c in res:
            assert c[0] == fe.FE_OK and c[2] <= 1e-8
    # the untrained network is Jacobi: the same iteration counts as PCG (within one)
    assert all(abs(a[1] - c[1]) <= 1 for a, c in zip(untrained, base))
    # the trained network needs fewer iterations than the method without it
    assert tot(trained) < tot(base), (tot(trained), tot(base))
    first.close()
    s.close()
    plain.close()


def test_harvest_in_mixed_precision_learned_context(fe):
    """A mixed-precision learned-solver context harvests one (b, x) pair per
    corrector through the plain-CG path (inner solves and refinement alike)."""
    import torch
    from paper_1404_0959_gb300 import learned
    N = 16
    rho, u, Y, T = random_fields(N, 1, False, seed=4, noise=0.0)
    s = fe.Solver([dict(N=N, nu=0.005, tau_p=[0.05], Y0=[0.01])], precision=fe.FE_FP32_MIXED,
                  solver=fe.FE_FCG_LEARNED, p_tol=1e-8)
    s.set_state(0, rho, u, Y)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(0))
    bank = learned.PairBank(s, 8)
    assert bank.harvest(s, 2) >= 4
    for k in range(bank.n):
        b, x = bank.b[k].double(), bank.x[k].double()
        assert torch.isfinite(b).all() and torch.isfinite(x).all()
        assert b.norm() > 0 and x.norm() > 0
    s.close()
