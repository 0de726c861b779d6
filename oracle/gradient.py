"""Adjoint gradient of the data misfit J(m) = 1/2 sum_s ||S u_s - d_s||^2
with respect to the squared slowness m (k^2 = omega^2 m), FP64.  Test
infrastructure only.

The method is the paper's Helmholtz operator (Sec. 2.1) with the adjoint
formed through the symmetrizer D (D A is symmetric, so A^H =
D conj(A) D^{-1}):  A^H lam = g  <=>  A x = conj(D^{-1} g), lam = D conj(x).
Only the diagonal of A depends on m:

    dA_nn / dm_n = -omega^2 - c_n * i * omega / (h * sqrt(m_n)),

with c_n the number of Sommerfeld sides of node n (0 interior, 1 edge,
2 corner; always 0 under Dirichlet boundaries), since each side adds
-2 i k / h to the centre and k = omega sqrt(m).  Then

    dJ/dm_n = - sum_s Re( conj(lam_s,n) * dA_nn/dm_n * u_s,n ).
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as ops


def sommerfeld_sides(level):
    ny, nx = level.ny, level.nx
    if level.bc != ops.SOMMERFELD:
        return np.zeros(level.n)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    c = ((ii == 0).astype(int) + (ii == nx - 1) + (jj == 0) + (jj == ny - 1))
    return c.ravel()[level.unk].astype(np.float64)


def diag_derivative(level, omega, m):
    """dA_nn/dm_n over the unknowns."""
    mu = np.asarray(m, np.float64).reshape(-1)[level.unk]
    c = sommerfeld_sides(level)
    return -omega ** 2 - c * 1j * omega / (level.h * np.sqrt(mu))


def misfit_and_gradient(nx, ny, h, m, omega, bc, sources, rec_idx, d_obs,
                        solve=None):
    """J and dJ/dm (full grid, zero on Dirichlet boundary nodes).

    ``sources``: (nshots, ny, nx) right-hand sides; ``rec_idx``: flat node
    indices of the receivers; ``d_obs``: (nshots, nrec) observed data.
    ``solve(A, rhs_unknowns) -> x`` defaults to a sparse LU solve.
    """
    m = np.asarray(m, np.float64).reshape(ny, nx)
    lv = ops.Level(nx, ny, h, omega ** 2 * m, bc)
    A = ops.five_point(lv, 1.0)
    if solve is None:
        lu = spla.splu(A.tocsc())
        solve = lambda _A, r: lu.solve(r)  # noqa: E731
    D = ops.symmetrizer(lv)
    ap = diag_derivative(lv, omega, m)
    rec_idx = np.asarray(rec_idx, dtype=np.int64)
    J = 0.0
    grad = np.zeros(lv.n)
    for s in range(len(sources)):
        u = solve(A, lv.to_unknowns(sources[s]))
        u_full = lv.to_full(u).reshape(-1)
        r = u_full[rec_idx] - d_obs[s]
        J += 0.5 * float(np.vdot(r, r).real)
        g_full = np.zeros(nx * ny, dtype=np.complex128)
        np.add.at(g_full, rec_idx, r)
        g = g_full[lv.unk]
        x = solve(A, np.conj(g / D))
        lam = D * np.conj(x)
        grad -= np.real(np.conj(lam) * ap * u)
    out = np.zeros(nx * ny)
    out[lv.unk] = grad
    return J, out.reshape(ny, nx)


def misfit(nx, ny, h, m, omega, bc, sources, rec_idx, d_obs):
    """J alone, by sparse LU solves (for finite-difference checks)."""
    m = np.asarray(m, np.float64).reshape(ny, nx)
    lv = ops.Level(nx, ny, h, omega ** 2 * m, bc)
    lu = spla.splu(ops.five_point(lv, 1.0).tocsc())
    J = 0.0
    for s in range(len(sources)):
        u_full = lv.to_full(lu.solve(lv.to_unknowns(sources[s]))).reshape(-1)
        r = u_full[np.asarray(rec_idx)] - d_obs[s]
        J += 0.5 * float(np.vdot(r, r).real)
    return J
