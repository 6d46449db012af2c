"""Discrete operators on the periodic uniform N^3 finite-volume grid (FP64).

Test infrastructure (see ``oracle/__init__``).

Grid: box [0, 2*pi)^3, N cells per side, spacing h = 2*pi/N, cell centres at
x_i = (i + 1/2) h.  Fields are numpy arrays of shape (N, N, N) indexed
[z, y, x], so the flat index is i + N*(j + N*k) with x fastest.  Direction
d = 0, 1, 2 means x, y, z, i.e. numpy axis 2 - d.  A face array F[d] holds
the value on the face between cell i and cell i + e_d ("face i+1/2").

Sec. 2 of the paper names the scheme only as "fourth order central
interpolation" inside a PISO finite-volume solver; the stencils below are the
reading adopted for it:

* I4  : 4-point fourth-order central interpolation to a face,
        (-f[i-1] + 9 f[i] + 9 f[i+1] - f[i+2]) / 16
* G4  : 4-point fourth-order face-normal gradient,
        (f[i-1] - 27 f[i] + 27 f[i+1] - f[i+2]) / (24 h)
* G2  : compact face-normal gradient (f[i+1] - f[i]) / h (pressure only)
* D   : finite-volume divergence of face values, sum_d (F[d][i] - F[d][i-e_d]) / h
* Gc  : Gauss cell gradient, (I4(f)[i+1/2] - I4(f)[i-1/2]) / h along d

Parity pins (tests/test_oracle_ops.py): each stencil applied to a sampled
Fourier mode equals its closed-form symbol; measured convergence order.
"""
import numpy as np


def axis(d):
    """numpy axis holding direction d (x fastest in memory)."""
    return 2 - d


def at(f, d, s):
    """Value of f at cell i + s*e_d for every cell i (periodic wrap)."""
    return np.roll(f, -s, axis=axis(d))


def I4(f, d):
    """Fourth-order central interpolation of cell field f to the d-faces."""
    return (-at(f, d, -1) + 9.0 * f + 9.0 * at(f, d, 1) - at(f, d, 2)) / 16.0


def G4(f, d, h):
    """Fourth-order face-normal gradient of cell field f on the d-faces."""
    return (at(f, d, -1) - 27.0 * f + 27.0 * at(f, d, 1) - at(f, d, 2)) / (24.0 * h)


def G2(f, d, h):
    """Compact second-order face-normal gradient on the d-faces."""
    return (at(f, d, 1) - f) / h


def Dd(F, d, h):
    """One-direction finite-volume difference of a d-face array to cells."""
    return (F - at(F, d, -1)) / h


def D(F, h):
    """Finite-volume divergence of the face vector F = (F[0], F[1], F[2])."""
    return Dd(F[0], 0, h) + Dd(F[1], 1, h) + Dd(F[2], 2, h)


def Gc(f, d, h):
    """Gauss cell gradient along d built from I4 face values."""
    return Dd(I4(f, d), d, h)


def stress(u, mu, h):
    """Viscous face stress tau[d][m] on the d-faces for velocity component m.

    tau_dm = mu * ( G4_d(u_m) + I4_d(Gc_m u_d) - 2/3 delta_dm I4_d(div u) ),
    div u = sum_l Gc_l u_l  (Newtonian, Stokes hypothesis, constant mu).
    """
    div = Gc(u[0], 0, h) + Gc(u[1], 1, h) + Gc(u[2], 2, h)
    tau = [[None] * 3 for _ in range(3)]
    for d in range(3):
        for m in range(3):
            t = G4(u[m], d, h) + I4(Gc(u[d], m, h), d)
            if d == m:
                t = t - (2.0 / 3.0) * I4(div, d)
            tau[d][m] = mu * t
    return tau


def div_stress(u, mu, h):
    """Cell divergence of the viscous stress: (D tau)_m for m = 0, 1, 2."""
    tau = stress(u, mu, h)
    return [D([tau[0][m], tau[1][m], tau[2][m]], h) for m in range(3)]


def L(u, phi, mu, h):
    """Momentum operator L_m(u, phi) = -D(phi_d I4_d(u_m)) + D(tau_dm).

    phi[d] is the mass flux per unit area on the d-faces.  Convection uses the
    fourth-order interpolated face velocity; diffusion the face stress above.
    """
    visc = div_stress(u, mu, h)
    out = []
    for m in range(3):
        conv = D([phi[d] * I4(u[m], d) for d in range(3)], h)
        out.append(-conv + visc[m])
    return out
