"""Write ``oracle_steps.json``: frozen outputs of the FP64 oracle on 8^3 cases.

The paper (arXiv:1404.0959) prints no worked example and no numeric result of
its solver, only the flow parameters (r.m.s. Mach 0.2 and 0.5, Sec. 1 and the
caption of Fig. 1).  The values stored here come from this script, which calls
``oracle/`` alone: the spectral initial field (seed 0, M 0.2, k0 2) with
deterministic density / temperature perturbations, two steps of Algorithm O
for each case, then the diagnostics.  They freeze the oracle: a later change
to its arithmetic shows up in ``tests/test_oracle_golden.py`` and must name
the passage that justifies it.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import diag, piso  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_steps.json")

CASES = {
    "barotropic": dict(closure=piso.BAROTROPIC),
    "fourier_3dust": dict(closure=piso.FOURIER, tau_p=[0.02, 0.1, 0.3], Y0=[0.02, 0.02, 0.02]),
    "transonic": dict(closure=piso.BAROTROPIC, transonic=True),
    "three_correctors": dict(closure=piso.BAROTROPIC, n_corr=3),
}


def case_state(prm):
    N = prm.N
    h = prm.h
    c = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    st = piso.initial_state(prm)
    rho = 1.0 + 0.05 * np.cos(x) * np.sin(2 * y) + 0.02 * np.cos(z)
    Y = [y0 * (1.0 + 0.1 * np.sin(x + j * z)) for j, y0 in enumerate(prm.Y0)]
    T = 1.0 + 0.03 * np.sin(x + z) if prm.closure == piso.FOURIER else None
    return piso.make_state(prm, rho, st["u"], Y, T)


def summarise(prm, st):
    h = prm.h
    d = diag.diagnostics(st["rho"], st["u"], h, nbins=4)
    tot = piso.totals(prm, st)
    return {
        "sum_rho": float(np.sum(st["rho"])),
        "l2_p": float(np.linalg.norm(st["p"])),
        "l2_u": [float(np.linalg.norm(c)) for c in st["u"]],
        "sum_rho_u": [float(np.sum(st["rho"] * c)) for c in st["u"]],
        "l2_phi": [float(np.linalg.norm(c)) for c in st["phi"]],
        "l2_Y": [float(np.linalg.norm(y)) for y in st["Y"]],
        "samples": {f"{i},{j},{k}": [float(st["rho"][i, j, k]), float(st["u"][0][i, j, k]),
                                     float(st["u"][1][i, j, k]), float(st["u"][2][i, j, k]),
                                     float(st["p"][i, j, k])]
                    for (i, j, k) in [(0, 0, 0), (1, 2, 3), (7, 5, 6), (4, 7, 0)]},
        "ke": d["ke"], "enstrophy": d["enstrophy"], "taylor": d["taylor"], "rho_rms": d["rho_rms"],
        "spectrum": [float(v) for v in d["spectrum"]],
        "mass": tot["mass"], "dust": tot["dust"], "energy": tot["energy"],
    }


def run_case(name):
    prm = piso.Params(N=8, k0=2.0, mach_rms=0.2, seed=0, **CASES[name])
    st = case_state(prm)
    out = {"params": {k: (v if not isinstance(v, float) or math.isfinite(v) else None)
                      for k, v in CASES[name].items()}, "steps": []}
    for _ in range(2):
        st, info = piso.step(prm, st)
        rec = summarise(prm, st)
        rec["dt"] = info["dt"]
        rec["iters"] = list(info["iters"])
        out["steps"].append(rec)
    return out


def main():
    data = {"source": "oracle/ (FP64), written by tests/golden/make_golden.py; the paper prints no "
                      "worked example (arXiv:1404.0959)",
            "cases": {name: run_case(name) for name in CASES}}
    with open(OUT, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


if __name__ == "__main__":
    main()
