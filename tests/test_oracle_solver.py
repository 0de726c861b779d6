"""Pins of the oracle's V-cycle, deflation, Krylov solvers and gradient."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from conftest import load_golden
from oracle import gradient as grd
from oracle import operators as ops
from oracle.krylov import gmres_left, gmres_right
from oracle.solver import Oracle


def _k2(ny, nx, seed, lo=3.0, hi=25.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(ny, nx)) ** 2


def _vcycle_matrix(orc, level):
    n = orc.levels[level].n
    B = np.zeros((n, n), dtype=complex)
    for c in range(n):
        e = np.zeros(n, dtype=complex)
        e[c] = 1.0
        B[:, c] = orc.vcycle(e, level)
    return B


@pytest.mark.parametrize("bc", [ops.SOMMERFELD, ops.DIRICHLET])
def test_vcycle_error_propagation_identity(bc):
    """Textbook multigrid identity, level by level:
    I - B_l M_l = S_l (I - P_l B_{l+1} R_l M_l) S_l with S_l = I - w D^-1 M_l,
    and B_L = M_L^{-1} at the coarsest level.  The weight is Sec. 3.1's
    relaxation parameter 0.8, written here rather than read from the oracle,
    so the identity also pins the weight the oracle's V-cycle uses by
    default."""
    nx, ny = 17, 9
    orc = Oracle(nx, ny, 0.05, _k2(ny, nx, 0), bc, z=None,
                 coarsest="direct")
    assert orc.L >= 2
    Bs = [_vcycle_matrix(orc, l) for l in range(orc.L + 1)]
    ML = orc.M[orc.L].toarray()
    np.testing.assert_allclose(Bs[orc.L] @ ML, np.eye(ML.shape[0]),
                               atol=1e-10)
    for l in range(orc.L):
        M = orc.M[l].toarray()
        n = M.shape[0]
        S = np.eye(n) - np.diag(0.8 / np.diag(M)) @ M
        P, R = orc.P[l].toarray(), orc.R[l].toarray()
        lhs = np.eye(n) - Bs[l] @ M
        rhs = S @ (np.eye(n) - P @ Bs[l + 1] @ R @ M) @ S
        np.testing.assert_allclose(lhs, rhs, atol=1e-10)


def test_coarsest_gmres_meets_its_tolerance():
    orc = Oracle(17, 17, 1 / 16, _k2(17, 17, 1), ops.SOMMERFELD, z=None)
    f = np.random.default_rng(2).standard_normal(orc.levels[-1].n) + 0j
    x = orc.coarsest_solve(f)
    r = np.linalg.norm(f - orc.M[-1] @ x) / np.linalg.norm(f)
    assert r <= 1e-8


@pytest.mark.parametrize("z,bc", [("bilinear", ops.DIRICHLET),
                                  ("ho", ops.SOMMERFELD),
                                  ("ho", ops.DIRICHLET)])
def test_deflation_invariants(z, bc):
    """With the Galerkin E solved exactly: P A Z = 0, R P = 0, Q A Z = Z and
    P_A-DEF1 A Z = Z for any M^{-1} (Sec. 3.2 definitions)."""
    nx, ny = 17, 13
    orc = Oracle(nx, ny, 0.04, _k2(ny, nx, 3), bc, z=z, e="galerkin",
                 coarse_tol=1e-14, coarse_maxit=400, coarsest="direct")
    A, Z, RZ = orc.A.toarray(), orc.Z.toarray(), orc.RZ.toarray()
    E = orc.E.toarray()
    Q = Z @ np.linalg.solve(E, RZ)
    Pd = np.eye(A.shape[0]) - A @ Q
    scale = np.abs(A @ Z).max()
    assert np.abs(Pd @ A @ Z).max() < 1e-10 * scale
    assert np.abs(RZ @ Pd).max() < 1e-10 * np.abs(RZ).max() * scale
    np.testing.assert_allclose(Q @ A @ Z, Z, atol=1e-10)
    # through the oracle's own inexact machinery at a tight tolerance
    rng = np.random.default_rng(4)
    c = rng.standard_normal(Z.shape[1]) + 1j * rng.standard_normal(Z.shape[1])
    v = A @ (Z @ c)
    np.testing.assert_allclose(orc.adef1(v), Z @ c, atol=1e-8 *
                               np.abs(Z @ c).max())


CASES = [
    (17, 17, ops.SOMMERFELD, "ho", "galerkin"),
    (17, 33, ops.DIRICHLET, "bilinear", "galerkin"),
    (17, 17, ops.SOMMERFELD, "ho", "red_glk2"),
    (17, 17, ops.DIRICHLET, "ho", "red_glk1"),
    (33, 17, ops.SOMMERFELD, "bilinear", "red_o2"),
    (17, 17, ops.SOMMERFELD, None, "galerkin"),
    (33, 33, ops.SOMMERFELD, "ho", "red_o4"),
    (33, 17, ops.DIRICHLET, "bilinear", "red_cmpo4"),
    (33, 33, ops.SOMMERFELD, "ho", "red_cmpo4"),
    (33, 33, ops.SOMMERFELD, "ho", "red_o6"),
    (33, 17, ops.DIRICHLET, "bilinear", "red_9pt"),
    (33, 33, ops.SOMMERFELD, "ho", "red_9pt"),
]


@pytest.mark.parametrize("nx,ny,bc,z,e", CASES)
def test_fgmres_matches_direct_solve(nx, ny, bc, z, e):
    h = 1.0 / (max(nx, ny) - 1)
    k2 = _k2(ny, nx, 5, lo=8, hi=20)
    orc = Oracle(nx, ny, h, k2, bc, z=z, e=e, coarse_tol=1e-10)
    rng = np.random.default_rng(6)
    b = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    x, info = orc.solve(b, tol=1e-12, maxit=200)
    lv = orc.levels[0]
    xd = lv.to_full(spla.spsolve(orc.A.tocsc(), lv.to_unknowns(b)))
    assert info.converged and info.relres < 1e-11
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_fgmres_warm_start_and_zero_rhs():
    orc = Oracle(17, 17, 1 / 16, _k2(17, 17, 7), ops.SOMMERFELD, z="ho")
    b = np.zeros((17, 17), complex)
    x, info = orc.solve(b)
    assert info.outer_iters == 0 and not np.any(x)
    b[8, 8] = 1.0
    x1, i1 = orc.solve(b, tol=1e-10)
    x2, i2 = orc.solve(b, tol=1e-10, x0_full=x1)
    assert i2.outer_iters <= 1 and i2.relres < 1e-9


@pytest.mark.parametrize("nx,ny,bc,z,e", CASES[:3])
def test_gcr_matches_direct_solve(nx, ny, bc, z, e):
    """Flexible GCR with A-DEF1 (Sec. 6.3's outer iteration) converges to
    the sparse-LU solution."""
    h = 1.0 / (max(nx, ny) - 1)
    k2 = _k2(ny, nx, 5, lo=8, hi=20)
    orc = Oracle(nx, ny, h, k2, bc, z=z, e=e, coarse_tol=1e-10)
    rng = np.random.default_rng(6)
    b = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    x, info = orc.solve_gcr(b, tol=1e-12, maxit=200)
    lv = orc.levels[0]
    xd = lv.to_full(spla.spsolve(orc.A.tocsc(), lv.to_unknowns(b)))
    assert info.converged and info.relres < 1e-11
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_gcr_equals_gmres_for_a_fixed_preconditioner():
    """With a fixed linear preconditioner P, GCR's directions span
    P K_k(A P, r0) and it minimises the residual over that space, as
    right-preconditioned GMRES does: the residual norms after k steps agree
    for every k (a property of the two methods, not of this code)."""
    from oracle.krylov import gcr_flexible
    n = 33
    orc = Oracle(n, n, 1 / 32, _k2(n, n, 9, lo=8, hi=20), ops.SOMMERFELD,
                 z="ho", coarsest="direct")
    lv = orc.levels[0]
    rng = np.random.default_rng(3)
    b = lv.to_unknowns(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))

    def prec(v):
        return orc.vcycle(v, 0)

    def matvec(v):
        return orc.A @ v

    for k in (1, 3, 6, 10):
        xg = gcr_flexible(matvec, b, 0.0, k, prec=prec).x
        xm = gmres_right(matvec, b, 0.0, k, prec=prec).x
        rg = np.linalg.norm(b - matvec(xg))
        rm = np.linalg.norm(b - matvec(xm))
        assert abs(rg - rm) <= 1e-9 * np.linalg.norm(b), (k, rg, rm)


def test_tlkm_converges_to_the_direct_solution():
    """FGMRES with the practical TLKM preconditioner converges to the
    sparse-LU solution (TLKM changes the convergence, not the system)."""
    n = 33
    k2 = _k2(n, n, 5, lo=8, hi=20)
    for bc, z in ((ops.SOMMERFELD, "ho"), (ops.DIRICHLET, "bilinear")):
        orc = Oracle(n, n, 1 / 32, k2, bc, z=z, coarse_tol=1e-10, precond="tlkm")
        rng = np.random.default_rng(8)
        b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        x, info = orc.solve(b, tol=1e-11, maxit=200)
        lv = orc.levels[0]
        xd = lv.to_full(spla.spsolve(orc.A.tocsc(), lv.to_unknowns(b)))
        assert info.converged and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_tlkm_with_exact_pieces_deflates_the_coarse_space():
    """With the exact pieces it approximates -- M~^-1 = M^-1 exactly and the
    coarse operator R_Z M^-1 A Z solved exactly -- TLKM with gamma = 1 maps
    the coarse space onto itself: P_TLKM A Z = Z (Sec. 3.2.2: P~ A~ Z =
    A~ Z - A~ Z + gamma Z).  Exercises the composition order of tlkm()."""
    n = 17
    orc = Oracle(n, n, 1 / 16, _k2(n, n, 2, lo=6, hi=12), ops.SOMMERFELD,
                 z="ho", coarsest="direct", precond="tlkm")
    lu = spla.splu(orc.M[0].tocsc())
    Minv = lambda v: lu.solve(v)  # noqa: E731
    Z = orc.Z.tocsc()
    coarse = orc.RZ @ np.column_stack(
        [Minv(orc.A @ Z[:, j].toarray().ravel()) for j in range(Z.shape[1])])
    orc.vcycle = lambda v, level=0: Minv(v)
    orc.coarse_solve_tlkm = lambda v1: np.linalg.solve(coarse, v1)
    for j in (0, 7, Z.shape[1] // 2, Z.shape[1] - 1):
        zj = Z[:, j].toarray().ravel().astype(complex)
        out = orc.tlkm(orc.A @ zj)
        assert np.linalg.norm(out - zj) <= 1e-9 * np.linalg.norm(zj), j


def test_table_b1_ordering_of_re_discretised_coarse_operators():
    """Appendix B's Table (129^2, k = 40, Dirichlet, centre source): ReD-O4
    needs the fewest outer iterations, ReD-9ptO2 next, ReD-O2 the most
    (paper: 14 / 15 / 17).  The counts themselves run about half the
    printed ones (as for the other re-discretised E, see the Table 5 rows),
    so only the ordering is pinned."""
    g = load_golden("red_o4_cmpo4_stencils.txt")["table_b1"]
    n, k = int(g[0, 0]), float(g[0, 1])
    assert list(g[0, 2:]) == [15, 17, 14]
    k2 = np.full((n, n), k * k)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    its = {}
    for e in ("red_9pt", "red_o2", "red_o4"):
        orc = Oracle(n, n, 1.0 / (n - 1), k2, ops.DIRICHLET, z="ho", e=e,
                     coarse_tol=1e-6)
        its[e] = orc.solve_left(b, tol=1e-6)[1].outer_iters
    assert its["red_o4"] <= its["red_9pt"] < its["red_o2"], its


E_COLS = ["galerkin", "red_o2", "red_o4", "red_cmpo4", "red_o6", "red_glk1",
          "red_glk2"]


def _table5_oracle(n, k):
    """Outer iterations and mean inner iterations per coarse solve of the
    oracle on a Table 5 row (left-preconditioned GMRES as in the paper)."""
    k2 = np.full((n, n), k * k)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    outer, inner = {}, {}
    for e in E_COLS:
        orc = Oracle(n, n, 1.0 / (n - 1), k2, ops.SOMMERFELD, z="ho", e=e,
                     coarse_tol=1e-6)
        info = orc.solve_left(b, tol=1e-6)[1]
        outer[e], inner[e] = info.outer_iters, float(np.mean(info.inner_iters))
    return outer, inner


def test_table5_comparisons_of_coarse_operators():
    """Table 5 (MP-2b, APD, kh = 0.625, 65^2 / k = 40 and 129^2 / k = 80)
    and the comparisons Sec. 6.2.2 draws from it.  Each comparison is
    checked on the printed numbers and on the oracle's counts:
    str-Glk needs the fewest outer iterations and the same number on both
    rows (+-1); ReD-O2 needs the most, more on the finer row; ReD-O4 needs
    fewer than ReD-O2 and ReD-O6 no fewer than ReD-O4; ReD-cmpO4 needs
    the fewest inner iterations per coarse solve among the re-discretised
    O-family; ReD-Glk1 and ReD-Glk2 keep their outer counts across the
    rows (+-1).  This runs the oracle at a coarse tolerance of 1e-6 with
    R_Z = Z^T / 4: its outer counts are lower than the printed ones for
    every re-discretised E (the printed scaling restores them), its inner
    counts about half (the printed ones are taken at 1e-12, pinned in
    test_table5_inner_counts_at_the_stated_coarse_tolerance); the paper's
    ReD-Glk1 > ReD-Glk2 does not hold here (7 / 8 on both rows), so it is
    not asserted."""
    g = load_golden("table5_mp2b.txt")
    rows = []
    for r in range(2):
        n, k = int(g["outer"][r, 0]), float(g["outer"][r, 1])
        paper = (dict(zip(E_COLS, g["outer"][r, 2:])),
                 dict(zip(E_COLS, g["inner"][r, 2:])))
        rows.append((paper, _table5_oracle(n, k)))
    for who in (0, 1):          # 0: printed, 1: oracle
        (o65, i65), (o129, i129) = (rows[0][who], rows[1][who])
        for o in (o65, o129):
            assert all(o["galerkin"] <= o[e] for e in E_COLS if o[e]), (who, o)
            assert all(o["red_o2"] >= o[e] for e in E_COLS), (who, o)
            assert o["red_o4"] < o["red_o2"], (who, o)
        assert abs(o65["galerkin"] - o129["galerkin"]) <= 1, who
        assert o129["red_o2"] > o65["red_o2"], who
        assert o129["red_o6"] >= o129["red_o4"], who
        for i in (i65, i129):
            assert all(i["red_cmpo4"] < i[e] for e in ("red_o2", "red_o4", "red_o6")
                       if i[e]), (who, i)
        for e in ("red_glk1", "red_glk2"):
            assert abs(o65[e] - o129[e]) <= 1, (who, e)


def _outer_printed(n, k, bc, z, e, precond):
    """Outer iterations of left-preconditioned GMRES (Alg. 1, 1e-6) with the
    deflation restriction as printed (R_Z = Z^T)."""
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), k * k), bc, z=z, e=e,
                 coarse_tol=1e-6, precond=precond, deflation_scaling="printed")
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    bu = orc.levels[0].to_unknowns(b)
    return gmres_left(lambda v: orc.A @ v, orc.precond, bu, 1e-6, 300).iters


def _near(ours, paper):
    return abs(ours - paper) <= max(2, round(0.1 * paper))


@pytest.mark.parametrize("table,row", [("table2", 0), ("table2", 1),
                                       ("table3", 0), ("table3", 1),
                                       ("table3", 2)])
def test_printed_scaling_reproduces_tables_2_and_3(table, row):
    """With the deflation restriction as the paper prints it (R_Z = Z^T,
    stencil sum 4, while ReD-O2 keeps the A_2h scale), the oracle's outer
    counts for A-DEF1 with str-Glk, A-DEF1 with ReD-O2 and the practical
    TLKM with ReD-O2 are the printed ones to +-2 (or 10 %)."""
    g = load_golden("outer_counts_tables_2_3.txt")[table][row]
    n, k = int(g[0]), float(g[1])
    bc = ops.DIRICHLET if table == "table2" else ops.SOMMERFELD
    ours = [_outer_printed(n, k, bc, "bilinear", e, pc)
            for e, pc in (("galerkin", "adef1"), ("red_o2", "adef1"),
                          ("red_o2", "tlkm"))]
    assert all(_near(o, int(p)) for o, p in zip(ours, g[2:])), (ours, g[2:])


@pytest.mark.parametrize("block", ["outer", "outer_kh03125"])
def test_printed_scaling_reproduces_table5_row(block):
    """Table 5, MP-2b, higher-order deflation vectors, 65^2 / k = 40
    (kh = 0.625) and 129^2 / k = 40 (kh = 0.3125, with ReD-O6): with
    R_Z = Z^T and the ReD-Glk 5x5 rows as printed, every coarse operator's
    outer count is the printed one to +-2, including ReD-Glk1 needing more
    iterations than ReD-Glk2 (its two ReD-O2 boundary rings are off the
    Z^T A Z scale, ReD-Glk2's one ring less so)."""
    g = load_golden("table5_mp2b.txt")[block][0]
    n, k = int(g[0]), float(g[1])
    ours = {e: _outer_printed(n, k, ops.SOMMERFELD, "ho", e, "adef1")
            for e, p in zip(E_COLS, g[2:]) if p}
    paper = {e: int(p) for e, p in zip(E_COLS, g[2:]) if p}
    assert all(_near(ours[e], paper[e]) for e in paper), (ours, paper)
    assert ours["red_glk1"] > ours["red_glk2"]


TABLE5_TAU_C = 1e-12   # Sec. 6, introduction: the coarse-grid solver's
                       # tolerance of the convergence study


def _table5_counts_printed(n, k, e):
    """Outer iterations and mean inner iterations per coarse solve of a
    Table 5 run: MP-2b, higher-order Z, left-preconditioned GMRES to 1e-6
    (Alg. 1), the coarse problem by CSLP-GMRES to the coarse tolerance the
    convergence study states (1e-12), deflation restriction as printed."""
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), k * k), ops.SOMMERFELD,
                 z="ho", e=e, coarse_tol=TABLE5_TAU_C,
                 deflation_scaling="printed")
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    info = orc.solve_left(b, tol=1e-6)[1]
    return info.outer_iters, float(np.mean(info.inner_iters))


@pytest.mark.parametrize("row,cols", [
    (0, ["galerkin", "red_o2", "red_o4", "red_cmpo4", "red_glk1", "red_glk2"]),
    (1, ["galerkin", "red_glk2"])])
def test_table5_inner_counts_at_the_stated_coarse_tolerance(row, cols):
    """Table 5's parenthesised counts (iterations of one coarse solve) are
    taken with the coarse-grid solver's tolerance at 1e-12, the value the
    introduction of Sec. 6 sets for the convergence study.  With that
    tolerance (and the printed deflation restriction, under which the
    outer counts are the printed ones) the oracle's mean inner iterations
    per coarse solve are the printed ones to within 20 % on the 65^2 row
    for every coarse operator and on the 129^2 row for str-Glk and
    ReD-Glk2 (measured ratios 0.93 ... 1.19; at a coarse tolerance of 1e-6
    they are about half).  A mistake in the coarse V-cycle, the CSLP
    shift, the coarse operators or the inner GMRES moves them off."""
    g = load_golden("table5_mp2b.txt")
    n, k = int(g["outer"][row, 0]), float(g["outer"][row, 1])
    po = dict(zip(E_COLS, g["outer"][row, 2:]))
    pi = dict(zip(E_COLS, g["inner"][row, 2:]))
    for e in cols:
        outer, inner = _table5_counts_printed(n, k, e)
        assert _near(outer, int(po[e])), (e, outer, po[e])
        assert 0.8 * pi[e] <= inner <= 1.2 * pi[e], (e, inner, pi[e])


def test_coarse_tolerance_study_sec63():
    """Sec. 6.3 / Table 9 on MP-2b 65^2, k = 40 (APD, ReD-Glk2):
    - the outer count of left-preconditioned GMRES does not depend on the
      coarse tolerance (Table 9's rows vary by at most one; so must ours);
    - its final true residual grows once the coarse tolerance is looser
      than the outer one, and stays put below it;
    - GCR keeps its count and reaches the 1e-6 residual at any coarse
      tolerance;
    - at tau_c = 0.1 the standard right-preconditioned GMRES, which assumes
      a fixed preconditioner, misses the residual target while flexible
      GMRES and GCR meet it."""
    rows = load_golden("iteration_tables.txt")["table9"]
    assert all(r.max() - r.min() <= 1 for r in rows)
    n, k = 65, 40.0
    k2 = np.full((n, n), k * k)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0

    def orc(tc):
        return Oracle(n, n, 1.0 / (n - 1), k2, ops.SOMMERFELD, z="ho",
                      e="red_glk2", coarse_tol=tc)

    left, gcr = {}, {}
    for tc in (1e-2, 1e-4, 1e-6, 1e-8):
        o = orc(tc)
        left[tc] = o.solve_left(b, tol=1e-6)[1]
        gcr[tc] = o.solve_gcr(b, tol=1e-6)[1]
    its = [i.outer_iters for i in left.values()]
    assert max(its) - min(its) <= 1, its
    assert left[1e-2].relres > 10 * left[1e-4].relres > 10 * left[1e-6].relres
    assert abs(left[1e-8].relres - left[1e-6].relres) <= 0.1 * left[1e-6].relres
    its = [i.outer_iters for i in gcr.values()]
    assert max(its) - min(its) <= 1 and all(i.relres <= 1e-6 for i in gcr.values())
    o = orc(1e-1)
    lv = o.levels[0]
    bu = lv.to_unknowns(b)
    std = gmres_right(lambda v: o.A @ v, bu, 1e-6, 200, prec=o.precond)
    assert std.converged
    assert np.linalg.norm(bu - o.A @ std.x) / np.linalg.norm(bu) > 1e-4
    assert o.solve(b, tol=1e-6)[1].relres <= 1e-6
    assert o.solve_gcr(b, tol=1e-6)[1].relres <= 1e-6


def test_three_level_deflation_invariant_and_direct_solution():
    """Three-level deflation: with the Galerkin level-2 operator and an
    exact level-2 solve, A-DEF1 of the level-1 system deflates its coarse
    space exactly (P_1 E Z_1 = Z_1, the eq. ADEF1 identity one level down);
    with ReD-Glk2 at level 2 the whole solve still reaches the direct
    solution."""
    n = 17
    k2 = _k2(n, n, 5, lo=6, hi=12)
    orc = Oracle(n, n, 1 / 16, k2, ops.SOMMERFELD, z="ho", coarsest="direct",
                 coarse_tol=1e-13, coarse_maxit=200, deflation_levels=2,
                 e2="galerkin")
    Z1 = orc.Z1.tocsc()
    for j in (0, Z1.shape[1] // 2, Z1.shape[1] - 1):
        zj = Z1[:, j].toarray().ravel().astype(complex)
        out = orc.adef1_level1(orc.E @ zj)
        assert np.linalg.norm(out - zj) <= 1e-9 * np.linalg.norm(zj), j
    for n, bc, z, kmax in ((17, ops.SOMMERFELD, "ho", 8.0),
                           (33, ops.DIRICHLET, "bilinear", 20.0)):
        k2 = _k2(n, n, 5, lo=0.4 * kmax, hi=kmax)
        orc = Oracle(n, n, 1.0 / (n - 1), k2, bc, z=z, coarse_tol=1e-8,
                     deflation_levels=2)
        rng = np.random.default_rng(12)
        b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        x, info = orc.solve(b, tol=1e-11, maxit=200)
        lv = orc.levels[0]
        xd = lv.to_full(spla.spsolve(orc.A.tocsc(), lv.to_unknowns(b)))
        assert info.converged and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_multilevel_deflation_invariant_and_direct_solution(depth):
    """Recursive A-DEF1 down to level D = depth.  (1) With Galerkin
    operators below level 1 (E_{l+1} = R_l E_l Z_l) and a tight solve of
    level l + 1 (the deepest one, D = l + 1), A-DEF1 of level l's coarse
    system deflates its coarse space exactly, P_l E_l Z_l = Z_l for
    l = D - 1 (the eq. ADEF1 identity l levels down).  (2) With ReD-Glk2 on
    every level below 1 and loose, capped inner solves at every level, a
    tight flexible-GMRES whole solve reaches the direct solution."""
    n = 33
    l = depth - 1
    k2 = _k2(n, n, 5, lo=6, hi=12)
    orc = Oracle(n, n, 1 / 32, k2, ops.SOMMERFELD, z="ho", coarsest="direct",
                 coarse_tol=1e-13, coarse_maxit=300, deflation_levels=depth,
                 e2="galerkin")
    assert sorted(orc.Ed) == list(range(1, depth + 1))
    Zl = orc.Zd[l].tocsc()
    for j in (0, Zl.shape[1] // 2, Zl.shape[1] - 1):
        zj = Zl[:, j].toarray().ravel().astype(complex)
        out = orc.adef1_at(l, orc.Ed[l] @ zj)
        assert np.linalg.norm(out - zj) <= 1e-9 * np.linalg.norm(zj), (l, j)
    k2 = _k2(n, n, 7, lo=8, hi=16)
    orc = Oracle(n, n, 1 / 32, k2, ops.SOMMERFELD, z="ho", coarse_tol=1e-1,
                 coarse_maxit=6, deflation_levels=depth)
    rng = np.random.default_rng(depth)
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x, info = orc.solve(b, tol=1e-11, maxit=200)
    lv = orc.levels[0]
    xd = lv.to_full(spla.spsolve(orc.A.tocsc(), lv.to_unknowns(b)))
    assert info.converged and np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_gmres_lucky_breakdown_identity():
    b = np.arange(1, 6) + 0j
    res = gmres_right(lambda v: 3.0 * v, b, 1e-14, 10)
    assert res.iters == 1
    np.testing.assert_allclose(res.x, b / 3.0)


def _band(paper, ours):
    return abs(ours - paper) <= max(2, 0.3 * paper)


def test_table2_band_mp2a_k20():
    """MP-2a, 33 x 33, k = 20, A-DEF1 str-Glk + CSLP-GMRES coarse solve:
    Table 2 prints 8 outer iterations (left preconditioning).  Plausibility
    band, both for Algorithm 1 and for the flexible GMRES used here."""
    g = load_golden("iteration_tables.txt")["table2_kh0625"]
    n, k, paper = (int(v) for v in g[0])
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), float(k) ** 2),
                 ops.DIRICHLET, z="bilinear", e="galerkin", coarse_tol=1e-6)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    _, il = orc.solve_left(b, tol=1e-6)
    _, ir = orc.solve(b, tol=1e-6)
    assert _band(paper, il.outer_iters), il.outer_iters
    assert _band(paper, ir.outer_iters), ir.outer_iters
    assert ir.relres <= 1e-6


@pytest.mark.parametrize("row", [0, 1])
def test_table3_band_mp2b(row):
    """MP-2b (Sommerfeld), bilinear str-Glk + CSLP-GMRES coarse solve:
    Table 3 prints 9 and 13 outer iterations for 33^2 / 65^2, kh = 0.625."""
    g = load_golden("iteration_tables.txt")["table3_kh0625"]
    n, k, paper = (int(v) for v in g[row])
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), float(k) ** 2),
                 ops.SOMMERFELD, z="bilinear", e="galerkin", coarse_tol=1e-6)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    _, il = orc.solve_left(b, tol=1e-6)
    assert _band(paper, il.outer_iters), il.outer_iters


@pytest.mark.slow
def test_config1_iterations_between_table2_rows():
    """81 x 81, k = 50, Dirichlet, bilinear str-Glk: the outer count lies
    between Table 2's k = 40 and k = 80 rows."""
    g = load_golden("iteration_tables.txt")["table2_kh0625"]
    lo, hi = int(g[1, 2]), int(g[2, 2])
    n = 81
    orc = Oracle(n, n, 1 / 80, np.full((n, n), 2500.0), ops.DIRICHLET,
                 z="bilinear", e="galerkin", coarse_tol=1e-6)
    b = np.zeros((n, n), complex)
    b[40, 40] = 1.0
    _, info = orc.solve(b, tol=1e-6)
    assert lo - 2 <= info.outer_iters <= hi + 2, info.outer_iters
    assert info.relres <= 1e-6


# ---------------------------------------------------------------- gradient
def _fd_setup(bc, nx=9, ny=13, seed=8):
    rng = np.random.default_rng(seed)
    h, omega = 1.0 / 12, 30.0
    m = rng.uniform(0.6, 1.4, size=(ny, nx))
    src = np.zeros((2, ny, nx), complex)
    src[0, ny // 2, nx // 2] = 1.0
    src[1, 2, 3] = 1.0
    row = 0 if bc == ops.SOMMERFELD else 1
    rec = (row * nx + np.arange(1, nx - 1)).astype(np.int64)
    d = (rng.standard_normal((2, rec.size))
         + 1j * rng.standard_normal((2, rec.size))) * 1e-3
    return nx, ny, h, m, omega, src, rec, d


@pytest.mark.parametrize("bc", [ops.SOMMERFELD, ops.DIRICHLET])
def test_gradient_matches_central_differences(bc):
    nx, ny, h, m, omega, src, rec, d = _fd_setup(bc)
    J, g = grd.misfit_and_gradient(nx, ny, h, m, omega, bc, src, rec, d)
    rng = np.random.default_rng(9)
    dirs = [rng.standard_normal((ny, nx)) for _ in range(3)]
    for (i, j) in ((4, 6), (0, 5), (0, 0), (8, 12)):   # interior/edge/corner
        e = np.zeros((ny, nx))
        e[j, i] = 1.0
        dirs.append(e)
    for dm in dirs:
        if bc == ops.DIRICHLET:
            dm = dm.copy()
            dm[0, :] = dm[-1, :] = dm[:, 0] = dm[:, -1] = 0.0
            if not np.any(dm):
                continue
        eps = 1e-4 * np.abs(m).max() / np.abs(dm).max()
        jp = grd.misfit(nx, ny, h, m + eps * dm, omega, bc, src, rec, d)
        jm = grd.misfit(nx, ny, h, m - eps * dm, omega, bc, src, rec, d)
        fd = (jp - jm) / (2 * eps)
        an = float(np.sum(g * dm))
        assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-30) + 1e-14, (fd, an)


def test_gradient_with_iterative_solves_matches_direct():
    nx, ny, h, m, omega, src, rec, d = _fd_setup(ops.SOMMERFELD, 9, 13)
    J0, g0 = grd.misfit_and_gradient(nx, ny, h, m, omega, ops.SOMMERFELD,
                                     src, rec, d)
    orc = Oracle(nx, ny, h, omega ** 2 * m, ops.SOMMERFELD, z="ho",
                 coarse_tol=1e-10, coarsest="direct")

    def it_solve(A, rhs):
        x, info = orc.solve(orc.levels[0].to_full(rhs), tol=1e-13)
        return orc.levels[0].to_unknowns(x)

    J1, g1 = grd.misfit_and_gradient(nx, ny, h, m, omega, ops.SOMMERFELD,
                                     src, rec, d, solve=it_solve)
    assert J1 == pytest.approx(J0, rel=1e-9)
    np.testing.assert_allclose(g1, g0, atol=1e-8 * np.abs(g0).max())
