"""Krylov solvers for the pressure-correction equation (FP64, textbook forms).

Test infrastructure (see ``oracle/__init__``).

Sec. 2 of the paper uses PISO, whose pressure-correction equation must be
solved each corrector; the paper does not name the linear solver.  Readings
adopted (standard algorithms, written from their textbook definitions):

* ``pcg``       Jacobi-preconditioned conjugate gradient (Hestenes-Stiefel),
                for the symmetric positive definite default operator; with
                ``precond`` any fixed symmetric positive definite
                preconditioner, e.g. ``neumann1``.
* ``neumann1``  first-order Neumann polynomial preconditioner
                P = D^-1 (2 I - M D^-1) (Dubois, Greenbaum and Rodrigue 1979,
                SIAM J. Numer. Anal. 16): the Neumann series of
                M^-1 = (I - (I - D^-1 M))^-1 D^-1 cut after its linear term,
                equivalently two Jacobi sweeps from zero.  Not the paper's
                (it names no preconditioner); symmetric positive definite
                because the eigenvalues of D^-1 M lie in (0, 2) for this
                strictly diagonally dominant operator.
* ``bicgstab``  Jacobi-preconditioned BiCGStab (van der Vorst 1992) for the
                non-symmetric "transonic" operator.
* ``fcg``       flexible CG (Notay 2000, truncation m_max = 1) for a
                preconditioner that changes from call to call (the learned
                one); a direction whose <z, r> is not positive falls back to
                the Jacobi direction.
* ``fgmres``    flexible GMRES(m) (Saad 1993, SIAM J. Sci. Comput. 14) for a
                changing preconditioner and any operator, the transonic one
                included: right preconditioning, Arnoldi with modified
                Gram-Schmidt, Givens rotations, restart after m directions; a
                preconditioner output that is not finite or is zero falls
                back to the Jacobi direction.

All four start from x = 0 and stop when the recurrence residual (for
``fgmres`` the least-squares residual of the Arnoldi relation) satisfies
||r||_2 <= tol ||b||_2; the returned ``rel_res_true`` is ||b - M x|| / ||b||
recomputed from x.  ||b|| == 0 returns x = 0 after zero iterations.

Parity pins (tests/test_oracle_solve.py): uniform psi against the exact
Fourier solution; variable psi on 8^3 against a dense LU solve of the matrix
assembled from the stencil coefficients; BiCGStab on the transonic operator
against its Fourier closed form; ``neumann1`` against two Jacobi sweeps, its
symmetry and the spectrum 1 - (1 - mu)^2 of P M for the eigenvalues mu of
D^-1 M (dense 6^3), PCG with it against the dense LU solve; flexible GMRES
against the same closed form,
and its defining property -- after k directions, x minimises ||b - M x|| over
the span of the k preconditioned directions -- against a least-squares solve
over an explicitly built basis.
"""
import numpy as np


def _norm(v):
    return float(np.sqrt(np.sum(v * v)))


def neumann1(matvec, diag):
    """The map v -> D^-1 (2 v - M (D^-1 v)) (first-order Neumann polynomial in D^-1 M)."""
    def apply(v):
        w = v / diag
        return (2.0 * v - matvec(w)) / diag
    return apply


def pcg(matvec, b, diag, tol, maxit, precond=None):
    """PCG with z = precond(r) (default Jacobi: z = r / diag).  Returns
    (x, iterations, rel_res_recurrence, rel_res_true)."""
    pre = precond if precond is not None else (lambda v: v / diag)
    x = np.zeros_like(b)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    z = pre(r)
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
        z = pre(r)
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


def _givens(a, b):
    """Rotation (c, s) with [c s; -s c] [a; b] = [hypot(a, b); 0]."""
    if b == 0.0:
        return 1.0, 0.0
    h = float(np.hypot(a, b))
    return a / h, b / h


def fgmres(matvec, b, precond, diag, tol, maxit, m=20, keep=0.9):
    """Flexible GMRES(m), right-preconditioned, x0 = 0.

    precond(v, it) returns the direction z_j for the unit Arnoldi vector v_j
    at overall iteration `it`, or None for the Jacobi direction v_j / diag
    (``precond`` None: always Jacobi).  A preconditioner direction is kept
    only if it is finite and non-zero, its image M z is not (to 1e-5 of its
    norm) in the span of the basis so far (which would make the Hessenberg
    matrix singular and the residual estimate meaningless), and its Arnoldi
    column shrinks the least-squares residual to at most ``keep`` times its
    previous value; otherwise the column is recomputed with the Jacobi
    direction (so a poor network cannot stall or fool the solve).  After each cycle of at most m
    directions, x += Z y with y the least-squares solution of the Hessenberg
    system; the next cycle starts from the true residual.  Same returns as
    ``pcg`` (the recurrence residual is the least-squares residual |g_{j+1}|).
    """
    x = np.zeros_like(b)
    bnorm = _norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, 0.0
    r = b.copy()
    it = 0
    res = bnorm
    while True:
        beta = _norm(r)
        if beta <= tol * bnorm:  # a restart's true residual already meets the tolerance
            res = beta
            break
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0

        def column(z, j):
            """Arnoldi column of direction z (modified Gram-Schmidt), its next
            basis vector, the column after the previous rotations, and ||M z||."""
            w = matvec(z)
            wn = _norm(w)
            h = np.zeros(j + 2)
            for i in range(j + 1):
                h[i] = float(np.sum(w * V[i]))
                w = w - h[i] * V[i]
            h[j + 1] = _norm(w)
            v = w / h[j + 1] if h[j + 1] > 0.0 else w
            for i in range(j):
                a, c = h[i], h[i + 1]
                h[i] = cs[i] * a + sn[i] * c
                h[i + 1] = -sn[i] * a + cs[i] * c
            return h, v, wn

        for j in range(m):
            z = precond(V[j], it) if precond is not None else None
            h = None
            if z is not None and np.all(np.isfinite(z)) and _norm(z) > 0.0:
                h, v, wn = column(z, j)
                c, s = _givens(h[j], h[j + 1])
                if not float(np.hypot(h[j], h[j + 1])) > 1e-5 * wn or abs(s) > keep:
                    h = None  # degenerate, or too little progress: the Jacobi direction instead
            if h is None:
                z = V[j] / diag
                h, v, _ = column(z, j)
            Z.append(z)
            V.append(v)
            H[: j + 2, j] = h
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            res = abs(g[j + 1])
            if res <= tol * bnorm or it >= maxit:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):  # back substitution on the rotated upper triangle
            y[i] = (g[i] - float(np.dot(H[i, i + 1:k], y[i + 1:k]))) / H[i, i]
        for i in range(k):
            x = x + y[i] * Z[i]
        if res <= tol * bnorm or it >= maxit:
            break
        r = b - matvec(x)
    true = _norm(b - matvec(x)) / bnorm
    return x, it, res / bnorm, true
