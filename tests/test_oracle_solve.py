"""Pins for the oracle's pressure-correction operator and Krylov solvers.

M p = psi p / dt - (dt/2) D(G2 p) (+ (1/2) D(I4(psi p) I4(HbyA)) transonic).
With uniform psi and HbyA the operator is diagonal in Fourier space; its
eigenvalues follow from the stencil symbols (2 sin(kh/2)/h for the compact
difference; Gc's symbol for D o I4).  For variable psi the matrix is
assembled here entry by entry from the 7-point stencil coefficients and
solved by dense LU.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from oracle import krylov, piso


def _rand(N, seed):
    return np.random.default_rng(seed).standard_normal((N, N, N))


def _fourier_solve(b, lam):
    return np.real(np.fft.ifftn(np.fft.fftn(b) / lam))


def _kgrid(N):
    kk = np.fft.fftfreq(N, d=1.0 / N)
    kz, ky, kx = np.meshgrid(kk, kk, kk, indexing="ij")
    return kx, ky, kz


def test_pcg_uniform_psi_matches_fourier():
    N, dt, psi0 = 16, 0.13, 0.83
    prm = piso.Params(N=N, p_tol=1e-14, p_maxit=400)
    h = prm.h
    psi = np.full((N, N, N), psi0)
    matvec, diag = piso.helmholtz(prm, psi, dt)
    b = _rand(N, 1)
    x, it, rec, true = krylov.pcg(matvec, b, diag, prm.p_tol, prm.p_maxit)
    K = _kgrid(N)
    lam = psi0 / dt + 0.5 * dt * sum(4 * np.sin(k * h / 2) ** 2 / h ** 2 for k in K)
    xe = _fourier_solve(b, lam)
    assert true < 1e-13
    assert np.max(np.abs(x - xe)) < 1e-12 * np.max(np.abs(xe))


def test_pcg_variable_psi_matches_dense_lu():
    N, dt = 8, 0.2
    prm = piso.Params(N=N, p_tol=1e-15, p_maxit=600)
    h = prm.h
    rng = np.random.default_rng(5)
    psi = 0.7 + 0.5 * rng.random((N, N, N))
    matvec, diag = piso.helmholtz(prm, psi, dt)
    b = rng.standard_normal((N, N, N))
    n = N ** 3
    A = np.zeros((n, n))
    off = -0.5 * dt / h ** 2

    def idx(i, j, k):
        return (i % N) + N * ((j % N) + N * (k % N))

    for k in range(N):
        for j in range(N):
            for i in range(N):
                r = idx(i, j, k)
                A[r, r] += psi[k, j, i] / dt + 3 * dt / h ** 2
                for (di, dj, dk) in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    A[r, idx(i + di, j + dj, k + dk)] += off
    xe = scipy.linalg.solve(A, b.reshape(-1)).reshape(N, N, N)
    x, it, rec, true = krylov.pcg(matvec, b, diag, 1e-14, 600)
    assert np.max(np.abs(x - xe)) < 1e-12 * np.max(np.abs(xe))
    # Jacobi diagonal equals the assembled diagonal
    np.testing.assert_allclose(diag.reshape(-1), np.diag(A), rtol=1e-15)


def test_bicgstab_transonic_matches_fourier():
    N, dt, psi0 = 16, 0.1, 0.9
    U = (0.3, -0.2, 0.15)
    prm = piso.Params(N=N, transonic=True)
    h = prm.h
    psi = np.full((N, N, N), psi0)
    HbyA = [np.full((N, N, N), U[d]) for d in range(3)]
    matvec, diag = piso.helmholtz(prm, psi, dt, HbyA)
    b = _rand(N, 2)
    x, it, rec, true = krylov.bicgstab(matvec, b, diag, 1e-14, 400)
    K = _kgrid(N)
    g = [(10 * np.sin(k * h) - np.sin(2 * k * h)) / (8 * h) for k in K]
    lam = psi0 / dt + 0.5 * dt * sum(4 * np.sin(k * h / 2) ** 2 / h ** 2 for k in K) \
        + 0.5 * psi0 * 1j * sum(U[d] * g[d] for d in range(3))
    xe = _fourier_solve(b, lam)
    assert true < 1e-13
    assert np.max(np.abs(x - xe)) < 1e-11 * np.max(np.abs(xe))


def test_fcg_with_jacobi_equals_pcg_solution():
    N, dt = 12, 0.17
    prm = piso.Params(N=N)
    rng = np.random.default_rng(9)
    psi = 0.8 + 0.3 * rng.random((N, N, N))
    matvec, diag = piso.helmholtz(prm, psi, dt)
    b = rng.standard_normal((N, N, N))
    x1, it1, _, t1 = krylov.pcg(matvec, b, diag, 1e-12, 500)
    x2, it2, _, t2 = krylov.fcg(matvec, b, lambda r: r / diag, diag, 1e-12, 500)
    assert t1 < 1e-12 and t2 < 1e-12
    # with a fixed SPD preconditioner FCG(1) is PCG in exact arithmetic
    assert abs(it1 - it2) <= 1
    assert np.max(np.abs(x1 - x2)) < 1e-10 * np.max(np.abs(x1))


def test_fcg_rejects_bad_direction():
    N, dt = 8, 0.2
    prm = piso.Params(N=N)
    psi = np.full((N, N, N), 1.0)
    matvec, diag = piso.helmholtz(prm, psi, dt)
    b = _rand(N, 4)
    # an adversarial "preconditioner" returning -r is replaced by Jacobi
    x, it, _, true = krylov.fcg(matvec, b, lambda r: -r, diag, 1e-12, 500)
    assert true < 1e-12


def test_zero_rhs():
    N = 8
    prm = piso.Params(N=N)
    matvec, diag = piso.helmholtz(prm, np.ones((N, N, N)), 0.1)
    x, it, rec, true = krylov.pcg(matvec, np.zeros((N, N, N)), diag, 1e-10, 10)
    assert it == 0 and not np.any(x)


def _transonic_system(N, dt, seed, variable=True):
    prm = piso.Params(N=N, transonic=True)
    rng = np.random.default_rng(seed)
    psi = 0.8 + 0.4 * rng.random((N, N, N)) if variable else np.full((N, N, N), 0.9)
    HbyA = [0.3 * rng.standard_normal((N, N, N)) for _ in range(3)]
    matvec, diag = piso.helmholtz(prm, psi, dt, HbyA)
    return matvec, diag, rng.standard_normal((N, N, N))


def test_fgmres_transonic_matches_fourier():
    """Flexible GMRES with Jacobi directions, restarted every 8, on the
    constant-coefficient transonic operator: the exact Fourier solution."""
    N, dt, psi0 = 16, 0.1, 0.9
    U = (0.3, -0.2, 0.15)
    prm = piso.Params(N=N, transonic=True)
    h = prm.h
    psi = np.full((N, N, N), psi0)
    HbyA = [np.full((N, N, N), U[d]) for d in range(3)]
    matvec, diag = piso.helmholtz(prm, psi, dt, HbyA)
    b = _rand(N, 2)
    x, it, rec, true = krylov.fgmres(matvec, b, None, diag, 1e-14, 400, m=8)
    K = _kgrid(N)
    g = [(10 * np.sin(k * h) - np.sin(2 * k * h)) / (8 * h) for k in K]
    lam = psi0 / dt + 0.5 * dt * sum(4 * np.sin(k * h / 2) ** 2 / h ** 2 for k in K) \
        + 0.5 * psi0 * 1j * sum(U[d] * g[d] for d in range(3))
    xe = _fourier_solve(b, lam)
    assert it > 8  # at least one restart
    assert true < 1e-13 and abs(rec - true) < 1e-12
    assert np.max(np.abs(x - xe)) < 1e-11 * np.max(np.abs(xe))


def _min_residual_over(matvec, b, Z):
    """argmin_{x in span Z} ||b - M x|| by least squares on the explicit basis."""
    MZ = np.stack([matvec(z).reshape(-1) for z in Z], axis=1)
    y, *_ = np.linalg.lstsq(MZ, b.reshape(-1), rcond=None)
    return sum(yi * z for yi, z in zip(y, Z))


@pytest.mark.parametrize("k", [1, 3, 7])
def test_fgmres_minimises_residual_over_its_directions(k):
    """The defining property of flexible GMRES: after k directions z_0..z_{k-1}
    (here an iteration-dependent preconditioner: Jacobi, identity, a damped
    Jacobi in turn), x_k minimises ||b - M x|| over their span.  Variable psi,
    non-symmetric transonic operator, 6^3."""
    matvec, diag, b = _transonic_system(6, 0.3, 7)
    seen = []

    def prec(v, it):
        z = [v / diag, v.copy(), 0.7 * v / diag + 0.1 * v][it % 3]
        seen.append(z)
        return z

    x, it, rec, true = krylov.fgmres(matvec, b, prec, diag, 0.0, k, m=20, keep=1.0)
    assert it == k and len(seen) == k
    xs = _min_residual_over(matvec, b, seen)
    assert np.max(np.abs(x - xs)) < 1e-9 * np.max(np.abs(xs))
    # the reported recurrence residual is the least-squares residual
    assert abs(rec - true) < 1e-12


def test_fgmres_jacobi_space_is_the_preconditioned_krylov_space():
    """With Jacobi directions only, x_k minimises the residual over
    D^{-1} K_k(M D^{-1}, b), built here power by power (k = 5)."""
    matvec, diag, b = _transonic_system(6, 0.3, 8)
    k = 5
    basis, v = [], b.copy()
    for _ in range(k):
        basis.append(v / diag)
        v = matvec(v / diag)
    x, it, _, _ = krylov.fgmres(matvec, b, None, diag, 0.0, k, m=20)
    xs = _min_residual_over(matvec, b, basis)
    assert np.max(np.abs(x - xs)) < 1e-8 * np.max(np.abs(xs))


def test_fgmres_restarts_and_falls_back():
    """Restarted every 4 directions, with a preconditioner that returns
    non-finite or zero directions on some calls (Jacobi is used there), the
    solve still reaches 1e-12 on the variable-psi transonic operator."""
    matvec, diag, b = _transonic_system(8, 0.2, 9)

    def prec(v, it):
        if it % 5 == 1:
            return np.full_like(v, np.nan)
        if it % 5 == 3:
            return np.zeros_like(v)
        return v / diag

    x, it, rec, true = krylov.fgmres(matvec, b, prec, diag, 1e-12, 500, m=4)
    assert true < 1e-12 * 1.01
    x0, _, _, _ = krylov.bicgstab(matvec, b, diag, 1e-14, 500)
    assert np.max(np.abs(x - x0)) < 1e-10 * np.max(np.abs(x0))
    z, it0, _, _ = krylov.fgmres(matvec, np.zeros_like(b), None, diag, 1e-12, 10)
    assert it0 == 0 and not np.any(z)


def test_fgmres_replaces_directions_that_make_no_progress():
    """Directions that add nothing are replaced by Jacobi's: one fixed vector
    returned every time (degenerate after its first use: its image is already
    in the basis), and fresh random vectors (non-degenerate but nearly
    useless).  Both solves converge in about the Jacobi-only iteration count;
    without the progress rule the random directions stall."""
    matvec, diag, b = _transonic_system(8, 0.2, 10)
    fixed = np.random.default_rng(11).standard_normal(b.shape)
    _, it_j, _, _ = krylov.fgmres(matvec, b, None, diag, 1e-12, 500, m=20)
    x, it, rec, true = krylov.fgmres(matvec, b, lambda v, k: fixed, diag, 1e-12, 500, m=20)
    assert true < 1e-12 * 1.01 and abs(rec - true) < 1e-12
    assert it <= it_j + 2
    rnd = np.random.default_rng(12)
    x, it, rec, true = krylov.fgmres(matvec, b, lambda v, k: rnd.standard_normal(v.shape), diag, 1e-12, 500, m=20)
    assert true < 1e-12 * 1.01 and it <= it_j + 4
    rnd = np.random.default_rng(12)
    _, it_s, rec_s, _ = krylov.fgmres(matvec, b, lambda v, k: rnd.standard_normal(v.shape), diag, 1e-12, 60,
                                      m=20, keep=1.0)
    assert it_s == 60 and rec_s > 1e-6


def _variable_system(N, dt, seed):
    prm = piso.Params(N=N)
    rng = np.random.default_rng(seed)
    psi = 0.6 + 0.6 * rng.random((N, N, N))
    matvec, diag = piso.helmholtz(prm, psi, dt)
    return matvec, diag, rng


def test_neumann1_is_two_jacobi_sweeps():
    # the first-order Neumann polynomial applied to b is the second Jacobi iterate for M x = b from x = 0
    matvec, diag, rng = _variable_system(10, 0.3, 21)
    b = rng.standard_normal((10, 10, 10))
    x = np.zeros_like(b)
    for _ in range(2):
        x = x + (b - matvec(x)) / diag
    y = krylov.neumann1(matvec, diag)(b)
    assert np.max(np.abs(y - x)) <= 1e-14 * np.max(np.abs(x))


def _dense(apply, N):
    n = N ** 3
    A = np.zeros((n, n))
    e = np.zeros(n)
    for j in range(n):
        e[j] = 1.0
        A[:, j] = apply(e.reshape(N, N, N)).reshape(-1)
        e[j] = 0.0
    return A


@pytest.mark.parametrize("dt", [0.05, 0.4])
def test_neumann1_symmetric_positive_with_squared_jacobi_spectrum(dt):
    N = 6
    matvec, diag, _ = _variable_system(N, dt, 22)
    M = _dense(matvec, N)
    P = _dense(krylov.neumann1(matvec, diag), N)
    assert np.max(np.abs(P - P.T)) <= 1e-13 * np.max(np.abs(P))
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0.0
    # D^-1 M is similar to the symmetric D^-1/2 M D^-1/2: eigenvalues mu in (0, 2)
    d = diag.reshape(-1)
    mu = np.sort(np.linalg.eigvalsh(M / np.sqrt(np.outer(d, d))))
    assert mu.min() > 0.0 and mu.max() < 2.0
    # I - P M = (I - D^-1 M)^2, so P M has the eigenvalues 1 - (1 - mu)^2, all in (0, 1]
    lam = np.sort(np.real(np.linalg.eigvals(P @ M)))
    np.testing.assert_allclose(lam, np.sort(1.0 - (1.0 - mu) ** 2), atol=1e-12)
    # the preconditioned condition number is below the Jacobi one
    assert lam.max() / lam.min() < mu.max() / mu.min()


def test_pcg_neumann1_matches_dense_lu_in_fewer_iterations():
    N, dt = 8, 0.4
    matvec, diag, rng = _variable_system(N, dt, 23)
    b = rng.standard_normal((N, N, N))
    xe = scipy.linalg.solve(_dense(matvec, N), b.reshape(-1)).reshape(N, N, N)
    xj, itj, _, tj = krylov.pcg(matvec, b, diag, 1e-13, 600)
    xp, itp, _, tp = krylov.pcg(matvec, b, diag, 1e-13, 600, precond=krylov.neumann1(matvec, diag))
    assert tp < 1e-13 and tj < 1e-13
    assert np.max(np.abs(xp - xe)) < 1e-12 * np.max(np.abs(xe))
    assert itp < itj
