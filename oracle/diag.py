"""Turbulence diagnostics (FP64).

Test infrastructure (see ``oracle/__init__``).

Sec. 2, par. 1 of the paper reports the energy spectrum, enstrophy, kinetic
energy and Taylor microscale; the caption of its Fig. 1 the non-dimensional
density r.m.s.  It gives no formulas.  Readings adopted (<.> = mean over
cells, derivatives by the Gauss cell gradient Gc of ``oracle.ops``):

* kinetic energy  KE   = <rho |u|^2> / 2   and  KE_u = <|u|^2> / 2
* enstrophy       Omega = <|curl u|^2> / 2
* Taylor microscale lambda = sqrt( sum_d <u_d^2> / sum_d <(Gc_d u_d)^2> )
* density r.m.s.  sqrt(<(rho - <rho>)^2>)
* spectrum        E(k) = sum over modes with round(|k|) = k of |u_hat|^2 / (2 N^6),
                  u_hat the unnormalised DFT, so sum_k E(k) = KE_u when every
                  shell is kept (Parseval).
* Q criterion     Q = (|Omega_ij|^2 - |S_ij|^2) / 2 from the Gc velocity gradient.

Parity pins (tests/test_oracle_diag.py): closed forms for a Taylor-Green
field (KE, enstrophy with the discrete gradient symbol, microscale), a single
Fourier mode in its shell, Parseval, density r.m.s. of a sine.
"""
import numpy as np

from . import ops


def grad(u, h):
    """g[m][l] = Gc_m(u_l): derivative along m of component l."""
    return [[ops.Gc(u[l], m, h) for l in range(3)] for m in range(3)]


def vorticity(u, h):
    g = grad(u, h)
    return [g[1][2] - g[2][1], g[2][0] - g[0][2], g[0][1] - g[1][0]]


def q_criterion(u, h):
    g = grad(u, h)
    s2 = 0.0
    w2 = 0.0
    for i in range(3):
        for j in range(3):
            # A_ij = du_i/dx_j = g[j][i]
            s = 0.5 * (g[j][i] + g[i][j])
            w = 0.5 * (g[j][i] - g[i][j])
            s2 = s2 + s * s
            w2 = w2 + w * w
    return 0.5 * (w2 - s2)


def spectrum(u, nbins):
    N = u[0].shape[0]
    kk = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    shell = np.floor(kmag + 0.5).astype(np.int64)
    dens = 0.0
    for c in range(3):
        uh = np.fft.fftn(u[c])
        dens = dens + (uh.real ** 2 + uh.imag ** 2)
    dens = dens / (2.0 * float(N) ** 6)
    e = np.zeros(nbins)
    mask = shell < nbins
    np.add.at(e, shell[mask], dens[mask])
    return e


def diagnostics(rho, u, h, nbins=0):
    usq = u[0] ** 2 + u[1] ** 2 + u[2] ** 2
    w = vorticity(u, h)
    num = float(np.mean(u[0] ** 2) + np.mean(u[1] ** 2) + np.mean(u[2] ** 2))
    den = float(sum(np.mean(ops.Gc(u[d], d, h) ** 2) for d in range(3)))
    out = {
        "ke": 0.5 * float(np.mean(rho * usq)),
        "ke_u": 0.5 * float(np.mean(usq)),
        "enstrophy": 0.5 * float(np.mean(w[0] ** 2 + w[1] ** 2 + w[2] ** 2)),
        "taylor": float(np.sqrt(num / den)) if den > 0 else 0.0,
        "rho_rms": float(np.sqrt(np.mean((rho - np.mean(rho)) ** 2))),
    }
    if nbins > 0:
        out["spectrum"] = spectrum(u, nbins)
    return out
