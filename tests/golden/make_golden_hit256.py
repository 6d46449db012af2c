"""Write ``hit256_step.json``: one FP64 oracle step at the benchmark size.

The workload is 256^3 decaying isotropic turbulence (barotropic, r.m.s. Mach
0.2 as in Sec. 1 and Fig. 1 of arXiv:1404.0959; k0 8, nu 0.001, one dust
class with tau_p 0.05 and Y 0.01, pressure residual 1e-8).  The paper prints
no numeric output, so this script, which calls ``oracle/`` alone, writes the
expected values: the spectral initial field (seed 0) rounded to FP32 (so that
an FP32 context can start from exactly the same numbers), one oracle step
from it, then full-field norms, totals, diagnostics and the values of every
state field at 1024 fixed cells.  The oracle step takes about two minutes
and 11 GB of host memory.

Run from the repository root:  python tests/golden/make_golden_hit256.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import diag, piso  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hit256_step.json")
N = 256
PARAMS = dict(N=N, nu=0.001, tau_p=[0.05], Y0=[0.01], mach_rms=0.2, k0=8.0, seed=0, p_tol=1e-8, p_maxit=1000)
NSAMPLE = 1024


def rounded_initial_state(prm):
    """The oracle's spectral initial state with every field rounded to FP32."""
    st = piso.initial_state(prm)
    r = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    return {"rho": r(st["rho"]), "u": [r(c) for c in st["u"]], "phi": [r(c) for c in st["phi"]],
            "p": r(st["p"]), "Y": [r(y) for y in st["Y"]], "T": None, "t": 0.0, "dt_prev": st["dt_prev"]}


def sample_cells():
    """Fixed (z, y, x) cells: the eight corners and faces' wrap cells plus a seeded draw."""
    edge = [(0, 0, 0), (0, 0, N - 1), (0, N - 1, 0), (N - 1, 0, 0), (N - 1, N - 1, N - 1),
            (127, 128, 255), (255, 31, 32), (1, 254, 2)]
    rng = np.random.default_rng(256)
    rest = rng.integers(0, N, size=(NSAMPLE - len(edge), 3))
    return [list(c) for c in edge] + rest.tolist()


def fields(st):
    out = {"rho": st["rho"], "p": st["p"]}
    for d in range(3):
        out["u%d" % d] = st["u"][d]
        out["phi%d" % d] = st["phi"][d]
    for j, y in enumerate(st["Y"]):
        out["Y%d" % j] = y
    return out


def main():
    prm = piso.Params(**PARAMS)
    st = rounded_initial_state(prm)
    new, info = piso.step(prm, st)
    cells = sample_cells()
    idx = tuple(np.array(cells).T)
    f = fields(new)
    d = diag.diagnostics(new["rho"], new["u"], prm.h)
    tot = piso.totals(prm, new)
    data = {
        "source": "oracle/ (FP64), written by tests/golden/make_golden_hit256.py; the paper prints no "
                  "worked example (arXiv:1404.0959)",
        "params": {k: v for k, v in PARAMS.items()},
        "initial": "oracle spectral initial state (seed 0) rounded to FP32",
        "dt": info["dt"], "iters": list(info["iters"]), "rel_res": list(info["rel_res"]),
        "cells_zyx": cells,
        "samples": {k: [float(v) for v in a[idx]] for k, a in f.items()},
        "l2": {k: float(np.linalg.norm(a)) for k, a in f.items()},
        "totals": {"mass": tot["mass"], "dust": tot["dust"], "energy": tot["energy"]},
        "diag": {k: d[k] for k in ("ke", "enstrophy", "taylor", "rho_rms")},
    }
    with open(OUT, "w") as fh:
        json.dump(data, fh, indent=0, sort_keys=True)
        fh.write("\n")


if __name__ == "__main__":
    main()
