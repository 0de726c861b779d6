"""GMRES variants with modified Gram-Schmidt Arnoldi and Givens rotations,
FP64 (Sec. 3.3, Algorithm 1).  Test infrastructure only.

``gmres_right``  right-preconditioned GMRES; with ``flexible=True`` the
                 preconditioned directions are kept (flexible GMRES, the
                 outer solver named in Sec. 6.3 for loose coarse
                 tolerances), otherwise the iterate is x0 + M^{-1} V y.
``gmres_left``   Algorithm 1: GMRES on the preconditioned operator,
                 stopping on the preconditioned relative residual.
``gcr_flexible`` the preconditioned Generalized Conjugate Residual method
                 with a variable right preconditioner (Sec. 3.3 names it,
                 after Eisenstat et al.; Sec. 6.3 uses it as the outer
                 iteration with a loose coarse tolerance).

Stopping rule of ``gmres_right``: after iteration j the Givens-updated
least-squares residual |g_{j+1}| is compared with ``tol * ||b||``.
"""

import numpy as np


class Result:
    def __init__(self, x, iters, res_est, converged):
        self.x = x
        self.iters = iters
        self.res_est = res_est
        self.converged = converged


def _givens(a, b):
    """Rotation (c real, s complex) with [c s; -conj(s) c] (a, b)^T = (r, 0)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, 1.0 + 0.0j
    t = np.sqrt(abs(a) ** 2 + abs(b) ** 2)
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def _arnoldi_lsq(apply_op, v0, beta, tol_abs, maxit, keep_dirs=None):
    """Shared Arnoldi/Givens loop.  ``apply_op(v) -> (w, z)`` returns the
    new Krylov vector w and (for flexible GMRES) the direction z."""
    n = v0.size
    V = [v0]
    Zs = []
    H = np.zeros((maxit + 1, maxit), dtype=np.complex128)
    g = np.zeros(maxit + 1, dtype=np.complex128)
    g[0] = beta
    cs = np.zeros(maxit)
    sn = np.zeros(maxit, dtype=np.complex128)
    k = 0
    res = beta
    for j in range(maxit):
        w, z = apply_op(V[j])
        if keep_dirs:
            Zs.append(z)
        for i in range(j + 1):                       # modified Gram-Schmidt
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        hn = np.linalg.norm(w)
        H[j + 1, j] = hn
        for i in range(j):                           # previous rotations
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
        H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        res = abs(g[j + 1])
        if res <= tol_abs or hn == 0.0:
            break
        V.append(w / hn)
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):                   # back substitution
        y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
    return V, Zs, y, k, res


def gmres_right(matvec, b, tol, maxit, x0=None, prec=None, flexible=False,
                restart=None):
    """Right-preconditioned (flexible) GMRES for matvec(x) = b.  With
    ``restart`` = m > 0 the Arnoldi process starts again from the true
    residual b - A x after every m iterations (GMRES(m)); the stopping test
    keeps the reference ||b||, and the count is the total over the cycles."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b) if x0 is None else np.asarray(x0, np.complex128).copy()
    bnorm = np.linalg.norm(b)
    prec = prec if prec is not None else (lambda v: v)

    def op(v):
        z = prec(v)
        return matvec(z), z

    total, res = 0, np.inf
    while True:
        r0 = b - matvec(x) if np.any(x) else b.copy()
        beta = np.linalg.norm(r0)
        if bnorm == 0.0 or beta <= tol * bnorm:
            return Result(x, total, beta, True)
        cycle = maxit - total
        if restart:
            cycle = min(cycle, restart)
        if cycle <= 0:
            return Result(x, total, res, False)
        V, Zs, y, k, res = _arnoldi_lsq(op, r0 / beta, beta, tol * bnorm, cycle,
                                        keep_dirs=flexible)
        if flexible:
            x = x + sum(y[i] * Zs[i] for i in range(k))
        else:
            x = x + prec(sum(y[i] * V[i] for i in range(k)))
        total += k
        if res <= tol * bnorm or not restart or k < cycle:
            return Result(x, total, res, res <= tol * bnorm)


def gmres_left(matvec, prec, b, tol, maxit, x0=None):
    """Algorithm 1 without the final deflation correction (which belongs to
    the singular P A formulation and is not used by A-DEF1): GMRES on
    prec(matvec(.)), stopping when the preconditioned residual falls below
    ``tol`` times the initial preconditioned residual."""
    b = np.asarray(b, dtype=np.complex128)
    x0 = np.zeros_like(b) if x0 is None else np.asarray(x0, np.complex128)
    r0 = prec(b - matvec(x0))
    beta = np.linalg.norm(r0)
    if beta == 0.0:
        return Result(x0.copy(), 0, 0.0, True)

    def op(v):
        return prec(matvec(v)), None

    V, _, y, k, res = _arnoldi_lsq(op, r0 / beta, beta, tol * beta, maxit)
    return Result(x0 + sum(y[i] * V[i] for i in range(k)), k, res,
                  res <= tol * beta)


def gcr_flexible(matvec, b, tol, maxit, x0=None, prec=None):
    """Flexible GCR: each step preconditions the current residual,
    u = P(r), c = A u, makes c orthogonal to the previous A-images by
    modified Gram-Schmidt (applying the same coefficients to u),
    normalises both by ||c||, and takes the step that minimises the
    residual along c: x += (c, r) u, r -= (c, r) c.  Stops when the
    recursively updated ||r|| <= tol ||b||."""
    x = np.zeros_like(b, dtype=np.complex128) if x0 is None else x0.astype(np.complex128)
    r = b - matvec(x) if x0 is not None else b.astype(np.complex128).copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return Result(np.zeros_like(x), 0, 0.0, True)
    U, Cs = [], []
    res = np.linalg.norm(r)
    k = 0
    while k < maxit and res > tol * bn:
        u = prec(r) if prec is not None else r.copy()
        c = matvec(u)
        for ci, ui in zip(Cs, U):
            beta = np.vdot(ci, c)
            c = c - beta * ci
            u = u - beta * ui
        a = np.linalg.norm(c)
        if a == 0.0:
            break
        c = c / a
        u = u / a
        gamma = np.vdot(c, r)
        x = x + gamma * u
        r = r - gamma * c
        Cs.append(c)
        U.append(u)
        res = np.linalg.norm(r)
        k += 1
    return Result(x, k, res, res <= tol * bn)
