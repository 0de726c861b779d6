"""Pins of the oracle's Krylov solvers (Sec. 3.3, Algorithm 1) by brute force
on tiny dense systems: the k-th iterate of each method is the minimiser of
its residual norm over its search space, which the tests build explicitly
and solve with a dense least-squares routine.  A wrong sign, a dropped
term, a swapped operand or a wrong rotation in the Arnoldi/Givens code
moves the iterate off that minimiser."""

import numpy as np
import pytest

from oracle.krylov import gcr_flexible, gmres_left, gmres_right

N = 12


def _system(seed):
    rng = np.random.default_rng(seed)
    A = (np.diag(4.0 + rng.random(N) + 1j * rng.random(N))
         + 0.4 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))))
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    x0 = 0.1 * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    # a fixed, non-trivial preconditioner (not an exact inverse)
    P = np.linalg.inv(np.diag(np.diag(A)) + 0.2 * np.tril(A, -1))
    return A, b, x0, P


def _krylov(op, r0, k):
    """Orthonormal basis of span{r0, op r0, ..., op^(k-1) r0}."""
    cols = [r0]
    for _ in range(k - 1):
        cols.append(op(cols[-1]))
    q, _ = np.linalg.qr(np.stack(cols, axis=1))
    return q


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("k", [1, 2, 4, 7])
def test_gmres_left_iterate_minimises_the_preconditioned_residual(k):
    """x_k = x0 + V y with V spanning K_k(P A, P r0), y minimising
    ||P (b - A x)||; the returned estimate is that minimum."""
    A, b, x0, P = _system(1)
    res = gmres_left(lambda v: A @ v, lambda v: P @ v, b, 0.0, k, x0=x0)
    assert res.iters == k
    r0 = P @ (b - A @ x0)
    V = _krylov(lambda v: P @ (A @ v), r0, k)
    y, *_ = np.linalg.lstsq(P @ A @ V, r0, rcond=None)
    x = x0 + V @ y
    assert _rel(res.x, x) < 1e-10
    assert abs(res.res_est - np.linalg.norm(P @ (b - A @ res.x))) < 1e-10 * np.linalg.norm(r0)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_gmres_right_iterate_minimises_the_true_residual(k):
    """Right preconditioning: x_k = x0 + P V y with V spanning K_k(A P, r0),
    y minimising ||b - A x||; the estimate is the true residual norm."""
    A, b, x0, P = _system(2)
    res = gmres_right(lambda v: A @ v, b, 0.0, k, x0=x0, prec=lambda v: P @ v)
    assert res.iters == k
    r0 = b - A @ x0
    V = _krylov(lambda v: A @ (P @ v), r0, k)
    y, *_ = np.linalg.lstsq(A @ P @ V, r0, rcond=None)
    x = x0 + P @ V @ y
    assert _rel(res.x, x) < 1e-10
    assert abs(res.res_est - np.linalg.norm(b - A @ res.x)) < 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("m,cycles", [(2, 2), (3, 3)])
def test_restarted_gmres_is_a_sequence_of_least_squares_cycles(m, cycles):
    """GMRES(m) (restart = m): after c cycles the iterate is x_c =
    x_{c-1} + P V y, V spanning K_m(A P, r_{c-1}) from the true residual
    r_{c-1} = b - A x_{c-1}, y minimising ||b - A x||; the count is c m."""
    A, b, x0, P = _system(5)
    res = gmres_right(lambda v: A @ v, b, 0.0, m * cycles, x0=x0,
                      prec=lambda v: P @ v, restart=m)
    assert res.iters == m * cycles
    x = x0.copy()
    for _ in range(cycles):
        r = b - A @ x
        V = _krylov(lambda v: A @ (P @ v), r, m)
        y, *_ = np.linalg.lstsq(A @ P @ V, r, rcond=None)
        x = x + P @ V @ y
    assert _rel(res.x, x) < 1e-10
    # more cycles than needed: the same as unrestarted GMRES once m >= N
    full = gmres_right(lambda v: A @ v, b, 1e-12, N, x0=x0, prec=lambda v: P @ v)
    big = gmres_right(lambda v: A @ v, b, 1e-12, N, x0=x0, prec=lambda v: P @ v,
                      restart=N)
    assert big.iters == full.iters and _rel(big.x, full.x) < 1e-12


class _Variable:
    """A preconditioner that changes with every application (two fixed
    matrices, alternating) and records its outputs."""

    def __init__(self, P1, P2):
        self.P = (P1, P2)
        self.calls = 0
        self.out = []

    def __call__(self, v):
        z = self.P[self.calls % 2] @ v
        self.calls += 1
        self.out.append(z)
        return z


@pytest.mark.parametrize("k", [2, 5])
def test_flexible_gmres_minimises_over_its_stored_directions(k):
    """Flexible GMRES with a variable preconditioner: x_k - x0 lies in the
    span of the preconditioned directions z_1..z_k it produced and
    minimises ||b - A x|| over that span."""
    A, b, x0, P = _system(3)
    pre = _Variable(P, np.eye(N) + 0.1 * P)
    res = gmres_right(lambda v: A @ v, b, 0.0, k, x0=x0, prec=pre, flexible=True)
    assert res.iters == k and len(pre.out) == k
    Z = np.stack(pre.out, axis=1)
    y, *_ = np.linalg.lstsq(A @ Z, b - A @ x0, rcond=None)
    assert _rel(res.x, x0 + Z @ y) < 1e-10


@pytest.mark.parametrize("k", [2, 5])
def test_flexible_gcr_minimises_over_its_preconditioned_residuals(k):
    """GCR with a variable preconditioner: x_k - x0 lies in the span of the
    preconditioned residuals P_i(r_i) and minimises ||b - A x|| over it
    (the A-images are orthonormal, so each step is the projection)."""
    A, b, x0, P = _system(4)
    pre = _Variable(P, np.eye(N) + 0.1 * P)
    res = gcr_flexible(lambda v: A @ v, b, 0.0, k, x0=x0, prec=pre)
    assert res.iters == k and len(pre.out) == k
    U = np.stack(pre.out, axis=1)
    y, *_ = np.linalg.lstsq(A @ U, b - A @ x0, rcond=None)
    assert _rel(res.x, x0 + U @ y) < 1e-10


def test_full_dimension_reaches_the_exact_solution():
    """After N steps every method has searched the whole space."""
    A, b, x0, P = _system(5)
    exact = np.linalg.solve(A, b)
    mv, pv = (lambda v: A @ v), (lambda v: P @ v)
    for x in (gmres_left(mv, pv, b, 0.0, N, x0=x0).x,
              gmres_right(mv, b, 0.0, N, x0=x0, prec=pv).x,
              gcr_flexible(mv, b, 0.0, N, x0=x0, prec=pv).x):
        assert _rel(x, exact) < 1e-9
