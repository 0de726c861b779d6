"""Pins of the oracle's operators against what the paper and the
mathematics fix (printed stencils, closed forms, invariants)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import load_golden
from oracle import operators as ops


def _rng_k2(ny, nx, seed, lo=5.0, hi=40.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(ny, nx)) ** 2


# ---------------------------------------------------------------- hierarchy
def test_level_shapes_rule():
    assert ops.level_shapes(81, 81) == [(81, 81), (41, 41), (21, 21),
                                        (11, 11), (6, 6)]
    assert ops.level_shapes(1281, 1281)[-1] == (6, 6)
    assert ops.level_shapes(2305, 769)[-1] == (10, 4)
    assert ops.level_shapes(289, 481)[-1] == (10, 16)
    assert ops.level_shapes(5, 5) == [(5, 5), (3, 3)]
    assert ops.level_shapes(2301, 751) == [(2301, 751), (1151, 376)]


def test_injection_of_wavenumber():
    k2 = _rng_k2(9, 17, 0)
    lv = ops.build_levels(17, 9, 0.1, k2, ops.SOMMERFELD)
    assert lv[1].k2[2, 3] == k2[4, 6]
    assert lv[1].h == pytest.approx(0.2)


# ---------------------------------------------------------------- A and M
@pytest.mark.parametrize("p,q", [(1, 1), (2, 3), (5, 1), (7, 7)])
def test_dirichlet_eigenpairs(p, q):
    """Appendix B: sin(p pi x) sin(q pi y) is an eigenvector of the Dirichlet
    5-point operator with h^-2 [4 - 2cos(p pi h) - 2cos(q pi h) - k^2 h^2]."""
    n, k = 9, 7.0
    h = 1.0 / (n - 1)
    lv = ops.Level(n, n, h, np.full((n, n), k * k), ops.DIRICHLET)
    A = ops.five_point(lv)
    x = np.arange(n) * h
    v = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
    lam = (4 - 2 * np.cos(p * np.pi * h) - 2 * np.cos(q * np.pi * h)
           - k * k * h * h) / h ** 2
    vu = lv.to_unknowns(v)
    np.testing.assert_allclose(A @ vu, lam * vu, atol=1e-10 * abs(lam))


def test_sommerfeld_rows_match_printed_stencils():
    g = load_golden("sommerfeld_stencils.txt")
    nx, ny, h = 7, 6, 0.05
    k2 = _rng_k2(ny, nx, 1)
    lv = ops.Level(nx, ny, h, k2, ops.SOMMERFELD)
    A = ops.five_point(lv).toarray()

    def row_stencil(i, j):
        r = A[j * nx + i]
        s = np.zeros((3, 3), dtype=complex)
        for dj, rr in ((1, 0), (0, 1), (-1, 2)):      # north, centre, south
            for di, cc in ((-1, 0), (0, 1), (1, 2)):  # west, centre, east
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    s[rr, cc] = r[jj * nx + ii]
        return s * h * h

    # left boundary point (i = 0, interior j), corner (0, 0) bottom-left
    for (i, j), key in (((0, 3), "edge"), ((0, 0), "corner")):
        s = row_stencil(i, j)
        expect = g[key].astype(complex)
        k = np.sqrt(k2[j, i])
        expect[1, 1] = 4 - k * k * h * h + g[key + "_c"][0, 0] * 1j * k * h
        np.testing.assert_allclose(s, expect, atol=1e-12)


def test_manufactured_solution_second_order():
    """Homogeneous variant of the commented-out closed-off problem (Sec. 2.2):
    u = sin(pi x) sin(2 pi y), b = (5 pi^2 - k^2) u, u = 0 on the boundary."""
    k = 10.0
    errs = []
    for n in (17, 33, 65, 129):
        h = 1.0 / (n - 1)
        lv = ops.Level(n, n, h, np.full((n, n), k * k), ops.DIRICHLET)
        x = np.arange(n) * h
        u = np.outer(np.sin(2 * np.pi * x), np.sin(np.pi * x))
        b = (5 * np.pi ** 2 - k * k) * u
        uh = spla.spsolve(ops.five_point(lv).tocsc(), lv.to_unknowns(b))
        errs.append(np.abs(uh - lv.to_unknowns(u)).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4.0) < 0.15), ratios


@pytest.mark.parametrize("bc", [ops.SOMMERFELD, ops.DIRICHLET])
def test_DA_symmetric(bc):
    nx, ny = 9, 13
    lv = ops.Level(nx, ny, 0.02, _rng_k2(ny, nx, 2), bc)
    A = ops.five_point(lv)
    DA = (np.diag(ops.symmetrizer(lv)) @ A.toarray())
    np.testing.assert_allclose(DA, DA.T, atol=1e-12 * np.abs(DA).max())
    if bc == ops.SOMMERFELD:
        assert np.abs(A.toarray() - A.toarray().T).max() > 1.0


@pytest.mark.parametrize("bc", [ops.SOMMERFELD, ops.DIRICHLET])
def test_cslp_minus_helmholtz_is_imaginary_mass(bc):
    """The CSLP of Sec. 5.1, ap = (4 - (beta1 - beta2 i) k^2 h^2)/h^2 with
    beta = (1, -0.5), differs from A by -0.5 i k^2 on the diagonal only:
    the same (negative) imaginary sign as the Sommerfeld rows' -2 i k / h."""
    from oracle.solver import Oracle
    nx, ny = 9, 7
    k2 = _rng_k2(ny, nx, 3)
    orc = Oracle(nx, ny, 0.03, k2, bc, z=None, coarsest="direct")
    d = (orc.M[0] - orc.A).toarray()
    np.testing.assert_allclose(d, np.diag(-0.5j * k2.ravel()[orc.levels[0].unk]),
                               atol=1e-9)
    if bc == ops.SOMMERFELD:
        lv = orc.levels[0]
        edge = lv.unk.tolist().index(3 * nx + 0)
        assert orc.A.diagonal()[edge].imag < 0


# ---------------------------------------------------------------- transfers
def _column_stencil(P, fine, coarse, I, J, r):
    col = P[:, J * coarse.nx + I].toarray().ravel()
    full = fine.to_full(col) if fine.n != fine.nx * fine.ny else \
        col.reshape(fine.ny, fine.nx)
    return full[2 * J - r:2 * J + r + 1, 2 * I - r:2 * I + r + 1].real


def test_bilinear_and_fw_match_printed():
    g = load_golden("transfer_stencils.txt")
    lv = ops.build_levels(17, 17, 0.1, np.ones((17, 17)), ops.SOMMERFELD)
    P = ops.prolongation(lv[0], lv[1], "bilinear")
    s = _column_stencil(P, lv[0], lv[1], 4, 3, 1)
    np.testing.assert_allclose(s, g["bilinear"] / g["bilinear_scale"][0, 0])
    R = ops.restriction(P)
    row = R[3 * lv[1].nx + 4].toarray().reshape(17, 17)[5:8, 7:10].real
    np.testing.assert_allclose(row, g["fw"] / g["fw_scale"][0, 0])


def test_ho_matches_printed_stencil_and_case_table():
    g = load_golden("transfer_stencils.txt")
    lv = ops.build_levels(17, 17, 0.1, np.ones((17, 17)), ops.SOMMERFELD)
    Z = ops.prolongation(lv[0], lv[1], "ho")
    s = _column_stencil(Z, lv[0], lv[1], 4, 4, 2)
    np.testing.assert_allclose(s, g["ho"] / g["ho_scale"][0, 0])
    # eq. (O4 matrix-free prolongation): the four node classes, 0-based with
    # the coarse node (ic, jc) on fine (2ic, 2jc)
    rng = np.random.default_rng(4)
    uc = rng.standard_normal((9, 9))
    uf = (Z @ uc.ravel()).reshape(17, 17).real
    for ic, jc in ((3, 4), (5, 2)):
        u = lambda a, b: uc[jc + b, ic + a]  # noqa: E731
        black = (6 * u(-1, 0) + 36 * u(0, 0) + 6 * u(1, 0) + u(-1, -1)
                 + 6 * u(0, -1) + u(1, -1) + u(-1, 1) + 6 * u(0, 1)
                 + u(1, 1)) / 64
        blue = (u(0, -1) + 6 * u(0, 0) + u(0, 1) + u(1, -1) + 6 * u(1, 0)
                + u(1, 1)) / 16
        red = (u(-1, 0) + 6 * u(0, 0) + u(1, 0) + u(-1, 1) + 6 * u(0, 1)
               + u(1, 1)) / 16
        grey = (u(0, 0) + u(0, 1) + u(1, 0) + u(1, 1)) / 4
        assert uf[2 * jc, 2 * ic] == pytest.approx(black, abs=1e-14)
        assert uf[2 * jc, 2 * ic + 1] == pytest.approx(blue, abs=1e-14)
        assert uf[2 * jc + 1, 2 * ic] == pytest.approx(red, abs=1e-14)
        assert uf[2 * jc + 1, 2 * ic + 1] == pytest.approx(grey, abs=1e-14)


@pytest.mark.parametrize("kind", ["bilinear", "ho"])
def test_transfers_reproduce_linear_functions(kind):
    lv = ops.build_levels(33, 17, 0.1, np.ones((17, 33)), ops.SOMMERFELD)
    Z = ops.prolongation(lv[0], lv[1], kind)
    Xc, Yc = np.meshgrid(np.arange(17) * 2.0, np.arange(9) * 2.0)
    uc = 0.3 + 1.7 * Xc - 0.6 * Yc
    Xf, Yf = np.meshgrid(np.arange(33) * 1.0, np.arange(17) * 1.0)
    uf = (Z @ uc.ravel()).reshape(17, 33).real
    inner = (slice(2, -2), slice(2, -2))
    np.testing.assert_allclose(uf[inner], (0.3 + 1.7 * Xf - 0.6 * Yf)[inner],
                               atol=1e-12)


# ---------------------------------------------------------------- Galerkin E
def _interior_row_stencil(E, lv, i, j, r):
    row = E[j * lv.nx + i].toarray().reshape(lv.ny, lv.nx)
    return row[j - r:j + r + 1, i - r:i + r + 1]


def test_galerkin_bilinear_closed_form():
    """Bilinear Galerkin of the 5-point operator, constant k, from the 1-D
    identities R1 L1 P1 = H^-2 [-1 2 -1] and R1 P1 = [1/8 3/4 1/8]."""
    n, h, k = 33, 1.0 / 32, 9.0
    lv = ops.build_levels(n, n, h, np.full((n, n), k * k), ops.SOMMERFELD)
    A = ops.five_point(lv[0])
    E = ops.galerkin(A, ops.prolongation(lv[0], lv[1], "bilinear"))
    H = 2 * h
    lap = np.array([[-0.25, -0.5, -0.25], [-0.5, 3.0, -0.5],
                    [-0.25, -0.5, -0.25]]) / H ** 2
    m1 = np.array([0.125, 0.75, 0.125])
    expect = lap - k * k * np.outer(m1, m1)
    np.testing.assert_allclose(_interior_row_stencil(E, lv[1], 8, 7, 1),
                               expect, atol=1e-9 * np.abs(expect).max())


def test_galerkin_ho_matches_printed_glk_stencils():
    """The explicit R A Z with the higher-order Z equals, on constant-k
    interior rows, ([Glk Laplace] - [ReD-Glk Kh]) / 4 as printed."""
    g = load_golden("glk_stencils.txt")
    n, h, k = 33, 1.0 / 32, 11.0
    lv = ops.build_levels(n, n, h, np.full((n, n), k * k), ops.SOMMERFELD)
    A = ops.five_point(lv[0])
    E = ops.galerkin(A, ops.prolongation(lv[0], lv[1], "ho"))
    H = 2 * h
    expect = (g["laplace"] / (g["laplace_scale"][0, 0] * H * H)
              - k * k * g["mass"] / g["mass_scale"][0, 0]) / 4.0
    got = _interior_row_stencil(E, lv[1], 8, 8, 2)
    np.testing.assert_allclose(got, expect, atol=1e-9 * np.abs(expect).max())
    # the re-discretised Glk stencil reproduces the same interior rows
    for variant in (1, 2):
        Eg = ops.red_glk(lv[1], variant)
        np.testing.assert_allclose(_interior_row_stencil(Eg, lv[1], 8, 8, 2),
                                   expect, atol=1e-9 * np.abs(expect).max())


def test_galerkin_ho_laplacian_taylor_expansion():
    """Sec. 5.2.4: -Lap_2h u = 4{-u_xx - u_yy - (13/48 u_xxxx + 1/2 u_xxyy +
    13/48 u_yyyy)(2h)^2} + O(h^4), exact for polynomials of degree <= 5
    (symmetric stencil: the remainder holds sixth derivatives only).  With
    R = Z^T/4 the operator is that expression divided by 4."""
    g = load_golden("glk_stencils.txt")
    a, b = g["taylor_a"][0, 0], g["taylor_b"][0, 0]
    n, h = 33, 0.05
    lv = ops.build_levels(n, n, h, np.zeros((n, n)), ops.SOMMERFELD)
    E = ops.galerkin(ops.five_point(lv[0]),
                     ops.prolongation(lv[0], lv[1], "ho"))
    X, Y = np.meshgrid(np.arange(17) * 2 * h, np.arange(17) * 2 * h)
    u = X ** 4 + 2 * X ** 2 * Y ** 2 - 3 * Y ** 4 + X ** 3 * Y + X * Y ** 2
    uxx = 12 * X ** 2 + 4 * Y ** 2 + 6 * X * Y
    uyy = 4 * X ** 2 - 36 * Y ** 2 + 2 * X
    uxxxx, uxxyy, uyyyy = 24.0, 8.0, -72.0
    expect = -uxx - uyy - (a * uxxxx + b * uxxyy + a * uyyyy) * (2 * h) ** 2
    got = (E @ u.ravel()).reshape(17, 17).real
    inner = (slice(3, -3), slice(3, -3))
    np.testing.assert_allclose(got[inner], expect[inner], rtol=1e-9,
                               atol=1e-8)


def test_ghost_rule_reproduces_sommerfeld_rows():
    """The ghost machinery used by ReD-Glk2, applied with the 5-point
    stencil, rebuilds the ghost-eliminated rows of eqs. (Sommerfeldstencil1/2)."""
    nx, ny, H = 8, 6, 0.07
    lv = ops.Level(nx, ny, H, _rng_k2(ny, nx, 5), ops.SOMMERFELD)
    inv = 1.0 / H ** 2

    def coef(i, j, di, dj, k2nb):
        if di == 0 and dj == 0:
            return 4 * inv - lv.k2[j, i]
        return -inv if abs(di) + abs(dj) == 1 else 0.0

    rows = np.ones((ny, nx), dtype=bool)
    S = ops.stencil_with_ghosts(lv, rows, coef, 1).toarray()
    A = ops.five_point_full(nx, ny, H, lv.k2, ops.SOMMERFELD).toarray()
    np.testing.assert_allclose(S, A, atol=1e-10 * np.abs(A).max())


def test_glk2_dirichlet_laplacian_sine_modes():
    """Under Dirichlet boundaries the ReD-Glk2 ghost (u_-1 = 2 u_0 - u_1 with
    u_0 = 0) is the odd reflection, so with k = 0 every unknown row applies
    the full 5x5 stencil to the odd extension: sine modes are eigenvectors
    with the stencil's Fourier symbol."""
    g = load_golden("glk_stencils.txt")
    n, H = 13, 1.0 / 12
    lv = ops.Level(n, n, H, np.zeros((n, n)), ops.DIRICHLET)
    E = ops.red_glk(lv, 2)
    S = g["laplace"] / (g["laplace_scale"][0, 0] * H * H) / 4.0
    x = np.arange(n) * H
    for p, q in ((1, 1), (3, 2), (6, 9)):
        v = np.outer(np.sin(q * np.pi * x), np.sin(p * np.pi * x))
        sym = sum(S[dy + 2, dx + 2] * np.cos(p * np.pi * H * dx)
                  * np.cos(q * np.pi * H * dy)
                  for dx in range(-2, 3) for dy in range(-2, 3))
        vu = lv.to_unknowns(v)
        np.testing.assert_allclose(E @ vu, sym * vu,
                                   atol=1e-9 * abs(S).max())


def test_glk2_sommerfeld_second_ring_rows_are_consistent():
    """ReD-Glk2's 5x5 rows on the second ring reach one layer of ghost nodes,
    filled by eq. (GhostPoint); the rows next to a corner also reach the
    corner ghost.  For a smooth u that satisfies the first-order Sommerfeld
    condition on every side (u = p(x) p(y) with -p'(0) = i k p(0) and
    p'(1) = i k p(1)), the Laplacian part of those rows must approximate
    -Lap u with an error that falls like H^2 under refinement, at an edge
    row and at the corner row alike.  The mass part takes ghost k^2 = 0
    (Sec. 5.2.4), so it is summed over the real nodes with the printed mass
    stencil and added back.  A corner ghost built with the wavenumber of a
    ghost node in its second application of eq. (GhostPoint) drops a
    2 i k H u term: its corner-row error then grows like 1/H."""
    g = load_golden("glk_stencils.txt")
    mass = g["mass"] / g["mass_scale"][0, 0] / 4.0
    k = 7.0
    a = -1j * k
    b = (2j * k + k * k) / (2 - 1j * k)

    def p(x):
        return 1 + a * x + b * x * x

    assert abs(-a - 1j * k * p(0.0)) < 1e-12
    assert abs((a + 2 * b) - 1j * k * p(1.0)) < 1e-10
    errs = {"corner": [], "edge": []}
    for n in (17, 33, 65):
        H = 1.0 / (n - 1)
        lv = ops.Level(n, n, H, np.full((n, n), k * k), ops.SOMMERFELD)
        x = np.arange(n) * H
        U = np.outer(p(x), p(x))
        EU = lv.to_full(ops.red_glk(lv, 2) @ lv.to_unknowns(U))
        for key, (i, j) in (("corner", (1, 1)), ("edge", (n // 2, 1))):
            m = sum(mass[dj + 2, di + 2] * k * k * U[j + dj, i + di]
                    for dj in range(-2, 3) for di in range(-2, 3)
                    if 0 <= i + di < n and 0 <= j + dj < n)
            exact = -2 * b * (p(x[j]) + p(x[i]))
            errs[key].append(abs(EU[j, i] + m - exact) / abs(exact))
    for key, e in errs.items():
        assert e[1] < e[0] / 3 and e[2] < e[1] / 3, (key, e)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("bc", [ops.DIRICHLET, ops.SOMMERFELD])
def test_red_glk_mass_part_takes_each_nodes_own_wavenumber(variant, bc):
    """Sec. 5.2.4 derives the ReD-Glk mass stencil for a constant k; with a
    variable k each of its entries takes k^2 of its own coarse node (our
    reading).  The stencil sums to 1 (it is R_Z Z for the higher-order Z,
    which reproduces constants), so on rows whose 5x5 stencil reaches only
    unknowns the mass part E(0) - E(k) maps u = 1/k^2 to exactly 1; taking
    the centre node's k^2 for every entry would not."""
    n, H = 17, 1.0 / 16
    rng = np.random.default_rng(11)
    k2 = 30.0 + 20.0 * rng.random((n, n))
    lv_k = ops.Level(n, n, H, k2, bc)
    lv_0 = ops.Level(n, n, H, np.zeros((n, n)), bc)
    mass = ops.red_glk(lv_0, variant) - ops.red_glk(lv_k, variant)
    u = lv_k.to_unknowns(1.0 / k2)
    out = lv_k.to_full(mass @ u)
    np.testing.assert_allclose(out[3:-3, 3:-3], 1.0, atol=1e-12)
    # the same rows of the constant-k operator: mass part = k^2 * (sum 1)
    lv_c = ops.Level(n, n, H, np.full((n, n), 40.0), bc)
    mc = ops.red_glk(lv_0, variant) - ops.red_glk(lv_c, variant)
    np.testing.assert_allclose(lv_c.to_full(mc @ lv_c.to_unknowns(np.ones((n, n))))[3:-3, 3:-3],
                               40.0, atol=1e-10)


def test_red_o2_is_coarse_helmholtz():
    k2 = _rng_k2(9, 9, 6)
    lv = ops.build_levels(17, 17, 0.1, np.kron(k2, np.ones((2, 2)))[:17, :17],
                          ops.SOMMERFELD)
    E = ops.red_o2(lv[1])
    direct = ops.five_point_full(9, 9, 0.2, lv[1].k2, ops.SOMMERFELD)
    np.testing.assert_allclose(E.toarray(), direct.toarray())


# ---------------------------------------------------------------- ReD-O4 / ReD-cmpO4
def _const_level(n, k, bc):
    H = 1.0 / (n - 1)
    return ops.Level(n, n, H, np.full((n, n), float(k) ** 2), bc)


def _full_row(mat, lv, i, j):
    """Row of node (i, j) of an operator over the unknowns, as a full-grid
    (ny, nx) array."""
    pos = {u: p for p, u in enumerate(lv.unk)}
    row = mat.getrow(pos[j * lv.nx + i]).toarray().ravel()
    return lv.to_full(row)


def test_red_o4_interior_row_is_the_printed_stencil():
    g = load_golden("red_o4_cmpo4_stencils.txt")
    w = g["o4_1d"][0] / g["o4_1d_scale"][0, 0]
    # the printed cross is -1 x the 1-D weights along x plus along y
    cross = np.zeros((5, 5))
    cross[2, :] -= w
    cross[:, 2] -= w
    np.testing.assert_allclose(cross * 12.0, g["o4_cross"], atol=1e-13)
    for bc in (ops.SOMMERFELD, ops.DIRICHLET):
        lv = _const_level(17, 7.0, bc)
        E = ops.red_o4(lv)
        row = _full_row(E, lv, 8, 8)
        H = lv.h
        want = np.zeros((17, 17), complex)
        want[6:11, 6:11] = g["o4_cross"] / (12.0 * H * H)
        want[8, 8] -= 49.0
        np.testing.assert_allclose(row, want, atol=1e-9 * np.abs(want).max())
        # rows within one node of the boundary are the ReD-O2 rows
        o2 = ops.five_point(lv)
        for (i, j) in ((1, 8), (8, 15), (1, 1)):
            np.testing.assert_allclose(_full_row(E, lv, i, j),
                                       _full_row(o2, lv, i, j), atol=1e-9)


def test_red_o4_is_fourth_order_on_a_smooth_function():
    """(-Lap - k^2) u for u = sin(pi x) sin(2 pi y) is (5 pi^2 - k^2) u; the
    O4 rows' error shrinks 16x per halving of H (the O2 rows' 4x)."""
    errs = []
    for n in (33, 65, 129):
        lv = _const_level(n, 5.0, ops.DIRICHLET)
        x = np.linspace(0.0, 1.0, n)
        u = np.sin(np.pi * x)[None, :] * np.sin(2 * np.pi * x)[:, None]
        got = lv.to_full(ops.red_o4(lv) @ lv.to_unknowns(u))
        exact = (5 * np.pi ** 2 - 25.0) * u
        inner = np.zeros((n, n), bool)
        inner[2:-2, 2:-2] = True
        errs.append(np.abs(got - exact)[inner].max())
    assert errs[0] / errs[1] > 14 and errs[1] / errs[2] > 14, errs


def test_red_cmpo4_coefficients_and_symbol():
    """The Singer-Turkel weights of Sec. 5.2.5 (fixture), their sums
    (sum a = 0: a Laplacian; sum b = 1: a mass average), and the operator
    on Dirichlet sine modes equals its closed-form symbol."""
    g = load_golden("red_o4_cmpo4_stencils.txt")
    a, b = ops.cmp_o4_weights(1.0)
    np.testing.assert_allclose(a, g["cmp_a"], atol=1e-15)
    np.testing.assert_allclose(b, g["cmp_b"], atol=1e-15)
    assert abs(a.sum()) < 1e-14 and abs(b.sum() - 1.0) < 1e-14
    n, k = 33, 9.0
    lv = _const_level(n, k, ops.DIRICHLET)
    E = ops.red_cmpo4(lv)
    H = lv.h
    x = np.linspace(0.0, 1.0, n)
    for p, q in ((1, 1), (3, 2), (7, 11)):
        u = np.sin(p * np.pi * x)[None, :] * np.sin(q * np.pi * x)[:, None]
        cx, cy = np.cos(p * np.pi * H), np.cos(q * np.pi * H)
        sa = a[1, 1] + 2 * a[1, 0] * (cx + cy) + 4 * a[0, 0] * cx * cy
        sb = b[1, 1] + 2 * b[1, 0] * (cx + cy) + 4 * b[0, 0] * cx * cy
        sym = sa / H ** 2 - sb * k * k
        got = E @ lv.to_unknowns(u)
        np.testing.assert_allclose(got, sym * lv.to_unknowns(u),
                                   atol=1e-9 * abs(sym))


def test_red_cmpo4_sommerfeld_ghost_rule():
    """At a left-edge Sommerfeld node the ghost column is eliminated with
    u_g = 2 i k H (1 - k^2 H^2 / 6) u_b + u_in (Sec. 5.2.5): the row acting
    on a vector equals the stencil applied to the vector extended by that
    rule, corner ghosts being the average of their two neighbouring edge
    ghosts."""
    n, kk = 9, 6.0
    lv = _const_level(n, kk, ops.SOMMERFELD)
    E = ops.red_cmpo4(lv)
    a, b = ops.cmp_o4_weights(1.0)
    H = lv.h
    rng = np.random.default_rng(4)
    u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ext = np.zeros((n + 2, n + 2), complex)
    ext[1:-1, 1:-1] = u
    c = 2j * kk * H * (1 - kk * kk * H * H / 6)
    ext[1:-1, 0] = c * u[:, 0] + u[:, 1]
    ext[1:-1, -1] = c * u[:, -1] + u[:, -2]
    ext[0, 1:-1] = c * u[0, :] + u[1, :]
    ext[-1, 1:-1] = c * u[-1, :] + u[-2, :]
    for (gj, gi, bj, bi) in ((0, 0, 1, 1), (0, -1, 1, -2), (-1, 0, -2, 1),
                             (-1, -1, -2, -2)):
        ext[gj, gi] = 0.5 * (ext[gj, bi] + ext[bj, gi])
    k2 = np.zeros((n + 2, n + 2))
    k2[1:-1, 1:-1] = kk * kk
    got = lv.to_full(E @ lv.to_unknowns(u))
    for (i, j) in ((0, 4), (0, 0), (4, 8), (8, 8)):
        want = 0.0
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                v = ext[j + 1 + dj, i + 1 + di]
                want += (a[dj + 1, di + 1] / H ** 2
                         - b[dj + 1, di + 1] * k2[j + 1 + dj, i + 1 + di]) * v
        assert abs(got[j, i] - want) <= 1e-10 * abs(want), (i, j)


def test_red_o6_weights_and_sixth_order():
    """ReD-O6 (Sec. 5.2.3): the printed weights, and on a smooth function
    the rows at least three nodes inside converge at sixth order (error
    ratio ~64 per halving of H; nodes nearer the boundary use ReD-O2)."""
    g = load_golden("red_o4_cmpo4_stencils.txt")
    w = g["o6_1d"][0] / g["o6_1d_scale"][0, 0]
    assert abs(w.sum()) < 1e-14
    # second moment of a second difference is 2 (d2/dx2 of x^2 / 2 ... = 1)
    x = np.arange(-3, 4)
    assert abs((w * x ** 2).sum() - 2.0) < 1e-13
    assert abs((w * x ** 4).sum()) < 1e-12 and abs((w * x ** 6).sum()) < 1e-11
    errs = []
    for n in (33, 65, 129):
        lv = _const_level(n, 5.0, ops.DIRICHLET)
        xs = np.linspace(0.0, 1.0, n)
        u = np.sin(np.pi * xs)[None, :] * np.sin(2 * np.pi * xs)[:, None]
        got = lv.to_full(ops.red_o6(lv) @ lv.to_unknowns(u))
        exact = (5 * np.pi ** 2 - 25.0) * u
        inner = np.zeros((n, n), bool)
        inner[3:-3, 3:-3] = True
        errs.append(np.abs(got - exact)[inner].max())
        # rows within two nodes of the boundary are the ReD-O2 rows
        o2 = ops.five_point(lv)
        for (i, j) in ((2, n // 2), (1, 1)):
            np.testing.assert_allclose(_full_row(ops.red_o6(lv), lv, i, j),
                                       _full_row(o2, lv, i, j), atol=1e-9)
    assert errs[0] / errs[1] > 50 and errs[1] / errs[2] > 50, errs


def test_red_9pt_coefficients_constraints_and_symbol():
    """ReD-9ptO2 (Appendix B): the printed coefficients meet the appendix's
    consistency constraints (a0 + 4 a_s + 4 a_c = 0, a_s + 2 a_c = -1,
    b0 + 4 b_s + 4 b_c = 1) to the printed digits, and the operator on
    Dirichlet sine modes equals the appendix's eigenvalue formula."""
    g = load_golden("red_o4_cmpo4_stencils.txt")
    a, b = ops.nine_point_o2_weights()
    np.testing.assert_allclose(a, g["ninept_a"], atol=1e-15)
    assert abs(a[1, 1] + 4 * a[1, 0] + 4 * a[0, 0]) < 1e-12
    assert abs(a[1, 0] + 2 * a[0, 0] + 1.0) < 1e-12
    assert abs(b.sum() - 1.0) < 1e-15
    n, k = 33, 9.0
    lv = _const_level(n, k, ops.DIRICHLET)
    E = ops.red_9pt(lv)
    H = lv.h
    xs = np.linspace(0.0, 1.0, n)
    for p, q in ((1, 2), (5, 5), (9, 14)):
        u = np.sin(p * np.pi * xs)[None, :] * np.sin(q * np.pi * xs)[:, None]
        cp, cq = np.cos(p * np.pi * H), np.cos(q * np.pi * H)
        lam = ((a[1, 1] - b[1, 1] * k * k * H * H)
               + 2 * (a[1, 0] - b[1, 0] * k * k * H * H) * (cp + cq)
               + 4 * (a[0, 0] - b[0, 0] * k * k * H * H) * cp * cq) / H ** 2
        np.testing.assert_allclose(E @ lv.to_unknowns(u), lam * lv.to_unknowns(u),
                                   atol=1e-9 * abs(lam))


def test_red_9pt_sommerfeld_uses_the_second_order_ghost_rule():
    n, kk = 9, 6.0
    lv = _const_level(n, kk, ops.SOMMERFELD)
    E = ops.red_9pt(lv)
    a, b = ops.nine_point_o2_weights()
    H = lv.h
    rng = np.random.default_rng(6)
    u = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    ext = np.zeros((n + 2, n + 2), complex)
    ext[1:-1, 1:-1] = u
    c = 2j * kk * H
    ext[1:-1, 0] = c * u[:, 0] + u[:, 1]
    ext[1:-1, -1] = c * u[:, -1] + u[:, -2]
    ext[0, 1:-1] = c * u[0, :] + u[1, :]
    ext[-1, 1:-1] = c * u[-1, :] + u[-2, :]
    for (gj, gi, bj, bi) in ((0, 0, 1, 1), (0, -1, 1, -2), (-1, 0, -2, 1),
                             (-1, -1, -2, -2)):
        ext[gj, gi] = 0.5 * (ext[gj, bi] + ext[bj, gi])
    got = lv.to_full(E @ lv.to_unknowns(u))
    for (i, j) in ((0, 4), (0, 0), (8, 8), (4, 4)):
        want = 0.0
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                inside = 0 <= i + di < n and 0 <= j + dj < n
                k2nb = kk * kk if inside else 0.0
                want += (a[dj + 1, di + 1] / H ** 2 - b[dj + 1, di + 1] * k2nb) \
                    * ext[j + 1 + dj, i + 1 + di]
        assert abs(got[j, i] - want) <= 1e-10 * abs(want), (i, j)
