"""A-priori analysis of the sub-grid stress for LES from resolved fields (FP64).

Test infrastructure (see ``oracle/__init__``).

Sec. 1 of the paper names large-eddy simulation of the gas-particle plume as
the goal its DNS serves, and Sec. 2 says the DNS database is meant for
a-priori tests of sub-grid models; it names no filter and no model.  Reading
adopted here:

* Filter: a top-hat of width Delta = 2 m h (m >= 1 cells either side) along
  each axis, integrated by the trapezoidal rule (end points at half weight),
  applied as a tensor product:
      fbar_i = (1 / 2m) [ f_{i-m}/2 + f_{i-m+1} + ... + f_{i+m-1} + f_{i+m}/2 ].
  Its transfer function per axis is
      G(k) = (1 / 2m) [ 1 + 2 sum_{l=1}^{m-1} cos(l k h) + cos(m k h) ].
* Favre (density-weighted) filtering for the compressible gas:
  rho_bar = bar(rho), u~_i = bar(rho u_i) / rho_bar.
* Sub-grid stress: tau_ij = bar(rho u_i u_j) - bar(rho u_i) bar(rho u_j) / rho_bar.
* Resolved strain from the method's own Gauss cell gradient Gc (ops.Gc):
  S_ij = (Gc_j u~_i + Gc_i u~_j) / 2, |S| = sqrt(2 S_ij S_ij).
* Model slot: Smagorinsky, B_ij = -2 rho_bar Delta^2 |S| S^d_ij (S^d the
  deviatoric strain), tau^M_ij = Cs^2 B_ij.
* Box statistics (means over the cells, tau^d the deviatoric stress):
      k_sgs   = <tau_kk> / 2                      sub-grid kinetic energy
      Pi      = -<tau^d_ij S_ij>                  sub-grid dissipation
      cs2_opt = <tau^d_ij B_ij> / <B_ij B_ij>      least-squares Cs^2
      corr    = <tau^d_ij B_ij> / sqrt(<tau^d:tau^d> <B:B>)
      Pi_M    = -Cs^2 <B_ij S_ij>                 model dissipation at Cs

Parity pins (tests/test_oracle_les.py): the filter's transfer function on
single modes against the closed form; the stress of a uniform flow is zero;
the stress of a single shear mode against its closed form; the model tensor
of a uniform strain against its closed form; Galilean invariance of tau.
"""
import numpy as np

from . import ops

# tensor components in the order (00, 01, 02, 11, 12, 22)
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def filter_weights(m):
    """Offsets -m..m and the trapezoidal top-hat weights of width 2 m h."""
    w = np.full(2 * m + 1, 1.0 / (2 * m))
    w[0] = w[-1] = 0.5 / (2 * m)
    return list(range(-m, m + 1)), w


def box_filter(f, m):
    """Tensor-product trapezoidal top-hat filter of width 2 m h (periodic)."""
    offs, w = filter_weights(m)
    out = f
    for d in range(3):
        g = np.zeros_like(out)
        for o, wo in zip(offs, w):
            g += wo * ops.at(out, d, o)
        out = g
    return out


def transfer(k, h, m):
    """Closed-form per-axis transfer function G(k) of the filter."""
    s = 1.0 + 2.0 * sum(np.cos(l * k * h) for l in range(1, m)) + np.cos(m * k * h)
    return s / (2 * m)


def filtered_fields(rho, u, m):
    """rho_bar, the Favre velocity u~ (3) and the stress tau (6, PAIRS order)."""
    rb = box_filter(rho, m)
    ru = [box_filter(rho * u[i], m) for i in range(3)]
    ut = [ru[i] / rb for i in range(3)]
    tau = [box_filter(rho * u[i] * u[j], m) - ru[i] * ru[j] / rb for i, j in PAIRS]
    return rb, ut, tau


def strain(ut, h):
    """Resolved strain S_ij (6, PAIRS order) from the Gauss cell gradient."""
    g = [[ops.Gc(ut[i], j, h) for j in range(3)] for i in range(3)]  # g[i][j] = Gc_j u~_i
    return [0.5 * (g[i][j] + g[j][i]) for i, j in PAIRS]


def _full(t6):
    """Component (i, j) of a symmetric tensor stored in PAIRS order."""
    idx = {(i, j): q for q, (i, j) in enumerate(PAIRS)}
    return lambda i, j: t6[idx[(min(i, j), max(i, j))]]


def contract(a6, b6):
    """a_ij b_ij summed over all nine components (symmetric tensors)."""
    out = 0.0
    for q, (i, j) in enumerate(PAIRS):
        out = out + (1.0 if i == j else 2.0) * a6[q] * b6[q]
    return out


def deviatoric(t6):
    tr = (t6[0] + t6[3] + t6[5]) / 3.0
    return [t6[q] - (tr if i == j else 0.0) for q, (i, j) in enumerate(PAIRS)]


def smagorinsky_tensor(rb, S, delta):
    """B_ij = -2 rho_bar Delta^2 |S| S^d_ij (the model is tau^M = Cs^2 B)."""
    mag = np.sqrt(2.0 * contract(S, S))
    Sd = deviatoric(S)
    return [-2.0 * rb * delta * delta * mag * s for s in Sd]


def apriori(rho, u, h, m, cs):
    """Box statistics of the a-priori test (see the module docstring)."""
    delta = 2 * m * h
    rb, ut, tau = filtered_fields(rho, u, m)
    S = strain(ut, h)
    B = smagorinsky_tensor(rb, S, delta)
    td = deviatoric(tau)
    tb = float(np.mean(contract(td, B)))
    bb = float(np.mean(contract(B, B)))
    tt = float(np.mean(contract(td, td)))
    return {
        "delta": delta,
        "k_sgs": 0.5 * float(np.mean(tau[0] + tau[3] + tau[5])),
        "pi_sgs": -float(np.mean(contract(td, S))),
        "cs2_opt": tb / bb if bb > 0 else 0.0,
        "corr": tb / np.sqrt(tt * bb) if tt > 0 and bb > 0 else 0.0,
        "pi_model": -cs * cs * float(np.mean(contract(B, S))),
    }
