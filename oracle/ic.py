"""Random solenoidal initial velocity with a prescribed energy spectrum (FP64).

Test infrastructure (see ``oracle/__init__``).

Sec. 1 of the paper studies freely decaying homogeneous isotropic turbulence
at r.m.s. Mach 0.2 or 0.5 but does not say how the initial field is made.
Reading adopted:

* Spectrum E(k) proportional to k^4 exp(-2 (k/k0)^2).
* For every FFT mode (flat index f = i + N*(j + N*k) in numpy's frequency
  order) and component c, a complex Gaussian g = (n1 + i n2)/sqrt(2) with
  (n1, n2) from Box-Muller on two uniforms.  The uniforms are outputs number
  m = 2*(3 f + c) and m + 1 of the SplitMix64 stream seeded with ``seed``.
* g is projected on the plane normal to k (solenoidal), scaled by
  sqrt(E(|k|) / (4 pi |k|^2)); the k = 0 mode and every mode with a Nyquist
  component are zeroed.
* u = Re(inverse 3D DFT), then rescaled so that sqrt(<|u|^2>) = M_rms
  (sound speed 1 at the reference state).

SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): output m of the stream with seed s is the mixing
function applied to s + (m + 1) * 0x9E3779B97F4A7C15 (mod 2^64); the mixer
is z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
z *= 0x94D049BB133111EB; z ^= z >> 31.  A uniform in (0, 1] is
((z >> 11) + 1) * 2^-53.

Parity pins (tests/test_oracle_ic.py): uniform and Gaussian moments within
sampling error, exact rescaled Mach number, spectral solenoidality of the
FFT of u, shell spectrum shape against E(k) within sampling error.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, m):
    """Output number m (array of uint64, 0-based) of the stream seeded with seed."""
    m = np.asarray(m, dtype=np.uint64)
    z = np.uint64(seed) + (m + np.uint64(1)) * GOLDEN
    z = (z ^ (z >> np.uint64(30))) * MIX1
    z = (z ^ (z >> np.uint64(27))) * MIX2
    return z ^ (z >> np.uint64(31))


def uniform01(z):
    """Map a uint64 draw to a double in (0, 1]."""
    return ((z >> np.uint64(11)).astype(np.float64) + 1.0) * 2.0 ** -53


def gaussian_pair(seed, m0):
    """Box-Muller on draws m0 and m0 + 1: returns (n1, n2), standard normals."""
    u1 = uniform01(splitmix64(seed, m0))
    u2 = uniform01(splitmix64(seed, np.asarray(m0, dtype=np.uint64) + np.uint64(1)))
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)


def wavenumbers(N):
    """Integer wavenumber per FFT index (numpy order), Nyquist as -N/2."""
    return np.fft.fftfreq(N, d=1.0 / N)


def spectrum_model(k, k0):
    """E(k) = k^4 exp(-2 (k/k0)^2) (unnormalised)."""
    return k ** 4 * np.exp(-2.0 * (k / k0) ** 2)


def spectral_velocity(N, k0, mach_rms, seed):
    """Random solenoidal velocity u[3] (each (N,N,N), [z,y,x]) with the model spectrum."""
    kk = wavenumbers(N)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    K = [kx, ky, kz]
    flat = np.arange(N ** 3, dtype=np.uint64).reshape(N, N, N)
    g = []
    for c in range(3):
        n1, n2 = gaussian_pair(seed, np.uint64(2) * (np.uint64(3) * flat + np.uint64(c)))
        g.append((n1 + 1j * n2) / np.sqrt(2.0))
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2safe = np.where(k2 > 0, k2, 1.0)
    kdotg = K[0] * g[0] + K[1] * g[1] + K[2] * g[2]
    kmag = np.sqrt(k2)
    amp = np.sqrt(spectrum_model(kmag, k0) / (4.0 * np.pi * k2safe))
    keep = k2 > 0
    if N % 2 == 0:
        nyq = -(N // 2)
        keep &= (kx != nyq) & (ky != nyq) & (kz != nyq)
    u = []
    for c in range(3):
        uh = (g[c] - K[c] * kdotg / k2safe) * amp
        uh = np.where(keep, uh, 0.0)
        u.append(np.real(np.fft.ifftn(uh)))
    ms = np.mean(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    scale = mach_rms / np.sqrt(ms)
    return [c * scale for c in u]
