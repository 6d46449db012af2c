"""Training and evaluation of the learned pressure preconditioner.

Orchestration only: the pairs come from the solver itself
(``fe_harvest_pressure``: right-hand side and converged correction of every
PISO corrector of a real run), and every forward pass, backward pass and Adam
update runs in the CUDA kernels of libfe.so (``fe_precond_train_step``).

Weights use the flat layout of ``include/fe.h``: per layer W[27][cin][cout]
then b[cout], layers e1a, e1b, d1, e2, d2, e3, u2, u1, out.
"""
import time

import numpy as np

from . import fe

LAYERS = [("e1a", 2, 16), ("e1b", 16, 16), ("d1", 16, 32), ("e2", 32, 32), ("d2", 32, 64), ("e3", 64, 64),
          ("u2", 96, 32), ("u1", 48, 16), ("out", 16, 1)]


def he_init(seed=0, zero_last=True):
    """He-normal weights (std sqrt(2 / (27 cin))), zero biases, flat layout.

    zero_last: the output layer starts at zero, so the untrained preconditioner
    is exactly the Jacobi direction (the network only corrects it)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, cin, cout in LAYERS:
        w = rng.standard_normal(27 * cin * cout) * np.sqrt(2.0 / (27 * cin))
        if zero_last and name == "out":
            w[:] = 0.0
        parts.append(w)
        parts.append(np.zeros(cout))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == fe.fe_preconditioner_size()
    return w


class PairBank:
    """Device buffers holding (b, x) pairs harvested from a running context,
    with the time step of the operator each pair belongs to."""

    def __init__(self, solver, capacity):
        import torch
        N = solver.N(0)
        self.b = [torch.empty((N, N, N), dtype=solver.dtype, device="cuda") for _ in range(capacity)]
        self.x = [torch.empty_like(self.b[0]) for _ in range(capacity)]
        self.dt = [0.0] * capacity
        self.n = 0

    def harvest(self, solver, steps):
        """Advance `steps` steps with the plain solver, keeping every corrector's pair."""
        for _ in range(steps):
            room = len(self.b) - self.n
            if room <= 0:
                break
            code, got = fe.fe_harvest_pressure(solver.ctx, [t.data_ptr() for t in self.b[self.n:]],
                                               [t.data_ptr() for t in self.x[self.n:]])
            if code != fe.FE_OK:
                raise fe.FeError(code, "fe_harvest_pressure")
            dt = solver.diagnostics(0)["dt_prev"]
            for k in range(self.n, self.n + got):
                self.dt[k] = dt
            self.n += got
        return self.n


def train(solver, bank, iters, lr=1e-3, log_every=0, first=0):
    """Cycle over the bank's pairs first..n-1 for `iters` Adam steps; returns the loss history."""
    hist = []
    t0 = time.perf_counter()
    span = bank.n - first
    for it in range(iters):
        k = first + it % span
        loss = fe.fe_precond_train_step(solver.ctx, 0, bank.b[k].data_ptr(), bank.x[k].data_ptr(), bank.dt[k], lr)
        hist.append(loss)
        if log_every and (it + 1) % log_every == 0:
            print("train %5d  loss %.4e  (%.1f s)" % (it + 1, loss, time.perf_counter() - t0), flush=True)
    return hist
