"""U-Net convolutions on the fifth-generation tensor cores (tcgen05, tensor
memory accumulators) against the warp-level MMA kernels, which the quantised
FP64 oracle pins (test_gpu_unet.py).

Both paths take BF16 operands and accumulate in FP32; they differ in the
order of the partial sums and therefore in occasional last-bit roundings of
the BF16 activations.  Bar: relative L2 <= 1e-2 per layer and on the output.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LAYERS = ["e1a", "e1b", "d1", "e2", "d2", "e3", "u2", "u1", "out"]
CH = [16, 16, 32, 32, 64, 64, 32, 16]
LEVEL = [0, 0, 1, 1, 2, 2, 1, 0]


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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def run(fe, N, mode, seed=0):
    import torch
    from paper_1404_0959_gb300 import learned
    s = fe.Solver([dict(N=N, nu=0.002, tau_p=[0.05], Y0=[0.01], mach_rms=0.2, k0=4.0, seed=1)],
                  precision=fe.FE_FP32_MIXED, solver=fe.FE_FCG_LEARNED, p_tol=1e-8)
    s.init_state(0, fe.FE_INIT_SPECTRAL)
    fe.fe_load_preconditioner(s.ctx, learned.he_init(seed, zero_last=False))
    fe.fe_precond_kernels(s.ctx, mode)
    g = torch.Generator(device="cuda").manual_seed(7)
    r = torch.randn(N, N, N, device="cuda", generator=g)
    z = torch.empty_like(r)
    fe.fe_precond_apply(s.ctx, 0, r.data_ptr(), 0.01, z.data_ptr())
    acts = {}
    for l in range(8):
        n = N >> LEVEL[l]
        if n <= 128:  # full-resolution activations of the 256^3 case stay on the device
            acts[l] = fe.fe_precond_activation(s.ctx, l, n ** 3 * CH[l])
    out = fe.fe_precond_activation(s.ctx, 8, N ** 3).astype(np.float64)  # the network output y
    s.close()
    return acts, out


@pytest.mark.parametrize("N", [128, 256])
def test_tensor_memory_convs_match_warp_mma(fe, N):
    a1, z1 = run(fe, N, 1)
    a0, z0 = run(fe, N, 0)
    errs = {LAYERS[l]: rel(a1[l], a0[l]) for l in a0}
    errs["out"] = rel(z1, z0)
    print("N=%d relative L2 tcgen05 vs warp MMA per layer:" % N, {k: "%.2e" % v for k, v in errs.items()})
    assert all(np.isfinite(v) for v in errs.values())
    bad = {k: v for k, v in errs.items() if not v <= 1e-2}
    assert not bad, errs
