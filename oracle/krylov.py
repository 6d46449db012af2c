"""Krylov solvers for the pressure-correction equation (FP64, textbook forms).

Test infrastructure (see ``oracle/__init__``).

Sec. 2 of the paper uses PISO, whose pressure-correction equation must be
solved each corrector; the paper does not name the linear solver.  Readings
adopted (standard algorithms, written from their textbook definitions):

* ``pcg``       Jacobi-preconditioned conjugate gradient (Hestenes-Stiefel),
                for the symmetric positive definite default operator.
* ``bicgstab``  Jacobi-preconditioned BiCGStab (van der Vorst 1992) for the
                non-symmetric "transonic" operator.
* ``fcg``       flexible CG (Notay 2000, truncation m_max = 1) for a
                preconditioner that changes from call to call (the learned
                one); a direction whose <z, r> is not positive falls back to
                the Jacobi direction.

All three start from x = 0 and stop when the recurrence residual satisfies
||r||_2 <= tol ||b||_2; the returned ``rel_res_true`` is ||b - M x|| / ||b||
recomputed from x.  ||b|| == 0 returns x = 0 after zero iterations.

Parity pins (tests/test_oracle_solve.py): uniform psi against the exact
Fourier solution; variable psi on 8^3 against a dense LU solve of the matrix
assembled from the stencil coefficients; BiCGStab on the transonic operator
against its Fourier closed form.
"""
import numpy as np


def _norm(v):
    return float(np.sqrt(np.sum(v * v)))


def pcg(matvec, b, diag, tol, maxit):
    """Jacobi-PCG.  Returns (x, iterations, rel_res_recurrence, rel_res_true)."""
    x = np.zeros_like(b)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    z = r / diag
    p = z.copy()
    rz = float(np.sum(r * z))
    it = 0
    rnorm = bnorm
    while it < maxit:
        q = matvec(p)
        alpha = rz / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rnorm = _norm(r)
        if rnorm <= tol * bnorm:
            break
        z = r / diag
        rz_new = float(np.sum(r * z))
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    true = _norm(b - matvec(x)) / bnorm
    return x, it, rnorm / bnorm, true


def bicgstab(matvec, b, diag, tol, maxit):
    """Right-Jacobi-preconditioned BiCGStab.  Same returns as ``pcg``."""
    x = np.zeros_like(b)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    rnorm = bnorm
    while it < maxit:
        rho = float(np.sum(rhat * r))
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = p / diag
        v = matvec(phat)
        alpha = rho / float(np.sum(rhat * v))
        s = r - alpha * v
        shat = s / diag
        t = matvec(shat)
        omega = float(np.sum(t * s)) / float(np.sum(t * t))
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        rho_old = rho
        it += 1
        rnorm = _norm(r)
        if rnorm <= tol * bnorm:
            break
    true = _norm(b - matvec(x)) / bnorm
    return x, it, rnorm / bnorm, true


def fcg(matvec, b, precond, diag, tol, maxit):
    """Flexible CG with one-vector truncation (Notay 2000).

    precond(r) returns a candidate direction z; if <z, r> <= 0 the Jacobi
    direction r / diag is used instead, so the method degrades to Jacobi-PCG
    rather than failing.  Same returns as ``pcg``.
    """
    x = np.zeros_like(b)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    p_prev = q_prev = None
    pq_prev = 0.0
    it = 0
    rnorm = bnorm
    while it < maxit:
        z = precond(r)
        if float(np.sum(z * r)) <= 0.0:
            z = r / diag
        if p_prev is None:
            p = z
        else:
            beta = float(np.sum(z * q_prev)) / pq_prev
            p = z - beta * p_prev
        q = matvec(p)
        pq = float(np.sum(p * q))
        alpha = float(np.sum(p * r)) / pq
        x = x + alpha * p
        r = r - alpha * q
        p_prev, q_prev, pq_prev = p, q, pq
        it += 1
        rnorm = _norm(r)
        if rnorm <= tol * bnorm:
            break
    true = _norm(b - matvec(x)) / bnorm
    return x, it, rnorm / bnorm, true
