"""Seeded synthetic inputs and the named workloads.

This module holds no arithmetic of the method: it only draws seeded random
fields (numpy) and lists workload parameters.  Tests feed the same arrays to
the CUDA path and to the FP64 oracle; the benchmark uses the workload table.

Workloads (decaying homogeneous isotropic turbulence, Sec. 1 of the paper:
r.m.s. Mach 0.2 / 0.5; 128^3 and 256^3 grids appear in the captions of its
Figs. 1 and 3):

``hit32``      32^3 FP64 barotropic, M 0.2, k0 4, nu 0.005, one dust class
               (Y 0.01, tau_p 0.05), 50 steps, CFL 0.5, Jacobi-PCG to 1e-10.
``hit128f``    128^3 Fourier (gamma 1.4, Pr 0.7), M 0.5, k0 4, nu 0.002,
               Y 0.05, tau_p 0.1, 200 steps; FP32 fields + FP64 reductions.
``hit256``     256^3 barotropic, M 0.2, k0 8, nu 0.001, tau_p 0.05, Y 0.01,
               500 steps, pressure residual 1e-8.
``ensemble64`` 64 independent barotropic FP32 boxes, N from {32,48,64,96},
               M from {0.2, 0.5}, tau_p uniform in [0.02, 0.5], seeds 0..63,
               nu 0.005, k0 4, Y 0.01, 100 steps.
``hit512f``    512^3 Fourier, M 0.5, k0 8, nu 5e-4, three dust classes
               (tau_p 0.02, 0.1, 0.3; Y 0.02 each), 1000 steps.
"""
import numpy as np

WORKLOADS = {
    "hit32": dict(N=32, closure=0, mach_rms=0.2, k0=4.0, nu=0.005, tau_p=[0.05], Y0=[0.01],
                  steps=50, cfl=0.5, p_tol=1e-10, precision="fp64", seed=0),
    "hit128f": dict(N=128, closure=1, gamma=1.4, Pr=0.7, mach_rms=0.5, k0=4.0, nu=0.002,
                    tau_p=[0.1], Y0=[0.05], steps=200, cfl=0.5, p_tol=1e-8, precision="mixed", seed=0),
    "hit256": dict(N=256, closure=0, mach_rms=0.2, k0=8.0, nu=0.001, tau_p=[0.05], Y0=[0.01],
                   steps=500, cfl=0.5, p_tol=1e-8, precision="mixed", seed=0),
    "hit512f": dict(N=512, closure=1, gamma=1.4, Pr=0.7, mach_rms=0.5, k0=8.0, nu=5e-4,
                    tau_p=[0.02, 0.1, 0.3], Y0=[0.02, 0.02, 0.02], steps=1000, cfl=0.5, p_tol=1e-8,
                    precision="mixed", seed=0),
}


def _splitmix64_first_uniform(seed):
    """First output of a SplitMix64 stream as a double in (0, 1] (input draw only)."""
    m = (1 << 64) - 1
    z = (seed + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    z ^= z >> 31
    return ((z >> 11) + 1) * 2.0 ** -53


def ensemble64_boxes(n_boxes=64):
    """Per-box parameters of the ensemble workload (box s uses seed s)."""
    boxes = []
    for s in range(n_boxes):
        boxes.append(dict(N=(32, 48, 64, 96)[s % 4], mach_rms=(0.2, 0.5)[(s // 4) % 2],
                          tau_p=[0.02 + 0.48 * _splitmix64_first_uniform(s)], Y0=[0.01],
                          nu=0.005, k0=4.0, seed=s, closure=0))
    return boxes


def smooth_field(N, seed, amp, kmax=4, mean=0.0):
    """Sum of random low-wavenumber cosines on the cell centres, [z, y, x] layout."""
    rng = np.random.default_rng(seed)
    h = 2 * np.pi / N
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    f = np.zeros((N, N, N))
    for _ in range(12):
        k = rng.integers(-kmax, kmax + 1, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.standard_normal() * np.cos(k[0] * x + k[1] * y + k[2] * z + ph)
    f *= amp / max(np.sqrt(np.mean(f * f)), 1e-300)
    return mean + f


def random_fields(N, n_dust, fourier, seed, mach=0.3, drho=0.05, noise=0.0):
    """Seeded state fields: rho, u[3], Y[n_dust], T (or None).

    Smooth random fields (a few low modes) plus optional white noise of
    relative size ``noise`` so that every stencil coefficient is exercised.
    """
    rng = np.random.default_rng(seed + 7919)
    rho = smooth_field(N, seed, drho, mean=1.0)
    u = [smooth_field(N, seed + 1 + d, mach / np.sqrt(3.0)) for d in range(3)]
    Y = [smooth_field(N, seed + 10 + j, 0.002, mean=0.01 * (j + 1)) for j in range(n_dust)]
    T = smooth_field(N, seed + 20, 0.03, mean=1.0) if fourier else None
    if noise > 0:
        rho = rho * (1 + noise * rng.standard_normal(rho.shape))
        u = [c + noise * mach * rng.standard_normal(c.shape) for c in u]
        Y = [y * (1 + noise * rng.standard_normal(y.shape)) for y in Y]
        if fourier:
            T = T * (1 + noise * rng.standard_normal(T.shape))
    return rho, u, Y, T


def random_vector(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N, N))
