"""GPU path (through the C ABI) against the CPU FP64 oracle, element by
element on seeded inputs.

Tolerances: FP64 operators 1e-12 relative (rounding-order differences
only); FP64 solves: outer iterations within +-1 of the oracle and, at tight
tolerances, solutions within 1e-8 relative; complex-FP32 preconditioner
operators 2e-5 relative (single-precision rounding of O(10) terms), and
mixed solves must still reach the FP64 residual target.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import gradient as grd
from oracle import operators as ops
from oracle.solver import Oracle
from paper_2308_06152_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2308_06152_gb300 import build
    build.build()


def solver(nx, ny, h, k2, bc, z="ho", e="galerkin", prec="fp64", nrhs=1,
           **kw):
    from paper_2308_06152_gb300.api import Desc, Solver
    return Solver(Desc(nx, ny, h, bc=bc, z=z, e=e, prec=prec, nrhs_max=nrhs,
                       **kw), k2)


def rk2(ny, nx, seed, lo=4.0, hi=30.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=(ny, nx)) ** 2


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_np(t):
    return t.cpu().numpy()


def oapply(orc, mat, lin, lout, x):
    return orc.levels[lout].to_full(mat @ orc.levels[lin].to_unknowns(x))


# ragged grid: 97 = 3*32 + 1 columns, 73 = 9*8 + 1 rows of 32x8 tiles
NX, NY = 97, 73
H = 1.0 / 96
BCS = ["sommerfeld", "dirichlet"]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_level_operators(bc, prec, tol):
    k2 = rk2(NY, NX, 1)
    s = solver(NX, NY, H, k2, bc, z="ho", prec=prec, nrhs=2)
    orc = Oracle(NX, NY, H, k2, bc, z="ho", coarsest="direct")
    assert s.num_levels == orc.L + 1
    for l in range(orc.L + 1):
        lv = orc.levels[l]
        assert s.level_shape(l) == (lv.nx, lv.ny)
        x = wl.random_complex((2, lv.ny, lv.nx), 10 + l)
        y = to_np(s.apply("cslp", x, l))
        for r in range(2):
            assert rel(y[r], oapply(orc, orc.M[l], l, l, x[r])) < tol
        if l < orc.L:
            y = to_np(s.apply("restrict_fw", x, l))
            assert rel(y[0], oapply(orc, orc.R[l], l, l + 1, x[0])) < tol
            lc = orc.levels[l + 1]
            xc = wl.random_complex((2, lc.ny, lc.nx), 20 + l)
            y = to_np(s.apply("prolong_bilinear", xc, l))
            assert rel(y[1], oapply(orc, orc.P[l], l + 1, l, xc[1])) < tol
    x = wl.random_complex((2, NY, NX), 3)
    y = to_np(s.apply("helmholtz", x))
    assert rel(y[1], oapply(orc, orc.A, 0, 0, x[1])) < 1e-12


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("z", ["bilinear", "ho"])
@pytest.mark.parametrize("e", ["galerkin", "red_o2", "red_glk1", "red_glk2",
                               "red_o4", "red_cmpo4", "red_o6", "red_9pt"])
def test_deflation_operators(bc, z, e):
    k2 = rk2(NY, NX, 2)
    s = solver(NX, NY, H, k2, bc, z=z, e=e)
    orc = Oracle(NX, NY, H, k2, bc, z=z, e=e, coarsest="direct")
    lc = orc.levels[1]
    x = wl.random_complex((1, NY, NX), 4)
    xc = wl.random_complex((1, lc.ny, lc.nx), 5)
    assert rel(to_np(s.apply("restrict_z", x))[0],
               oapply(orc, orc.RZ, 0, 1, x[0])) < 1e-12
    assert rel(to_np(s.apply("prolong_z", xc))[0],
               oapply(orc, orc.Z, 1, 0, xc[0])) < 1e-12
    assert rel(to_np(s.apply("coarse_e", xc))[0],
               oapply(orc, orc.E, 1, 1, xc[0])) < 1e-12


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("z", ["bilinear", "ho"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
def test_stored_galerkin_stencil(bc, z, prec, tol):
    """stcl-op-Glk: the Galerkin product's per-node stencil, extracted at
    setup by FP64 probing, applied to several right-hand sides against the
    oracle's explicit R_Z A Z (FP64 to 1e-12; FP32-stored coefficients and
    FP32 arithmetic to 2e-6, below the on-the-fly FP32 product's error), by
    the one-node and the two-nodes-per-thread kernels (the coarse grid's
    odd row count leaves a half-filled pair in the last tile row)."""
    k2 = rk2(NY, NX, 2)
    s = solver(NX, NY, H, k2, bc, z=z, e="galerkin", prec=prec, nrhs=3)
    orc = Oracle(NX, NY, H, k2, bc, z=z, e="galerkin", coarsest="direct")
    lc = orc.levels[1]
    xc = wl.random_complex((3, lc.ny, lc.nx), 15)
    for rpb, pairs in ((0, 0), (2, 0), (1, 0), (0, 1), (2, 1), (1, 1)):
        s.set_tuning(galerkin_apply=1, e_rhs_per_block=rpb, e_column_pairs=pairs)
        y = to_np(s.apply("coarse_e", xc))
        for r in range(3):
            assert rel(y[r], oapply(orc, orc.E, 1, 1, xc[r])) < tol, (rpb, pairs, r)
    s.set_tuning(galerkin_apply=0)
    y0 = to_np(s.apply("coarse_e", xc))
    assert rel(y0[0], oapply(orc, orc.E, 1, 1, xc[0])) < max(tol, 2e-5)


def test_stored_galerkin_stencil_rejected_without_galerkin_e():
    from paper_2308_06152_gb300.api import HzError
    s = solver(NX, NY, H, rk2(NY, NX, 2), "sommerfeld", z="ho", e="red_glk2")
    with pytest.raises(HzError):
        s.set_tuning(galerkin_apply=1)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 5e-5)])
def test_vcycle(bc, prec, tol):
    k2 = rk2(NY, NX, 6)
    s = solver(NX, NY, H, k2, bc, z="ho", prec=prec)
    orc = Oracle(NX, NY, H, k2, bc, z="ho", coarsest="direct")
    for l in (0, 1, orc.L):
        lv = orc.levels[l]
        f = wl.random_complex((1, lv.ny, lv.nx), 30 + l)
        y = to_np(s.apply("vcycle", f, l))[0]
        ref = lv.to_full(orc.vcycle(lv.to_unknowns(f[0]), l))
        assert rel(y, ref) < tol, (l, rel(y, ref))


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 5e-5),
                                      ("mixed_bf16", 2e-2)])
def test_fused_vcycle_matches_oracle(bc, prec, tol):
    """The fused smoothing/transfer kernels (vcycle_fused = 1) and their
    staged multi-RHS form (vcycle_fused = 2, with groups of right-hand sides
    that leave a ragged last group, both prolongation tiles) give the same
    V-cycle as the oracle from levels 0, 1 and L; the fused and staged
    kernels match the unfused ones to rounding (the staged ones form the
    residual as (1 - w) f + off-diagonal terms, with D^-1 diag(M) = w)."""
    k2 = rk2(NY, NX, 6)
    s = solver(NX, NY, H, k2, bc, z="ho", prec=prec, nrhs=3)
    orc = Oracle(NX, NY, H, k2, bc, z="ho", coarsest="direct")
    for l in (0, 1, orc.L):
        lv = orc.levels[l]
        f = wl.random_complex((3, lv.ny, lv.nx), 30 + l)
        s.set_tuning(vcycle_fused=0)
        y0 = to_np(s.apply("vcycle", f, l))
        s.set_tuning(vcycle_fused=1)
        y1 = to_np(s.apply("vcycle", f, l))
        for r in range(3):
            ref = lv.to_full(orc.vcycle(lv.to_unknowns(f[r]), l))
            assert rel(y1[r], ref) < tol, (l, r, rel(y1[r], ref))
            # unfused BF16 storage rounds x + P xc once more
            bound = {"fp64": 1e-13, "mixed": 1e-6, "mixed_bf16": 2e-2}[prec]
            assert rel(y1[r], y0[r]) < bound
        for rpb, tile in ((2, 0), (1, 1), (0, 1), (16, 0)):
            s.set_tuning(vcycle_fused=2, vcycle_rhs_per_block=rpb, vcycle_tile=tile)
            y2 = to_np(s.apply("vcycle", f, l))
            for r in range(3):
                ref = lv.to_full(orc.vcycle(lv.to_unknowns(f[r]), l))
                assert rel(y2[r], ref) < tol, (l, rpb, tile, r, rel(y2[r], ref))
                assert rel(y2[r], y0[r]) < bound, (l, rpb, tile, r)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 5e-5),
                                      ("mixed_bf16", 2e-2)])
def test_staged_vcycle_interior_tiles_match_oracle(bc, prec, tol):
    """On a grid large enough for tiles away from the boundary (257 x 97:
    the staged restriction and the 64 x 16 prolongation blocks then take
    their test-free interior path, the ragged edge tiles the general one),
    the staged V-cycle matches the oracle's from levels 0 and 1 and the
    unfused kernels to rounding."""
    nx, ny = 257, 97
    h = 1.0 / (nx - 1)
    k2 = rk2(ny, nx, 7)
    s = solver(nx, ny, h, k2, bc, z="ho", prec=prec, nrhs=3)
    orc = Oracle(nx, ny, h, k2, bc, z="ho", coarsest="direct")
    bound = {"fp64": 1e-13, "mixed": 1e-6, "mixed_bf16": 2e-2}[prec]
    for l in (0, 1):
        lv = orc.levels[l]
        f = wl.random_complex((3, lv.ny, lv.nx), 40 + l)
        s.set_tuning(vcycle_fused=0)
        y0 = to_np(s.apply("vcycle", f, l))
        for rpb, tile in ((2, 1), (0, 0)):
            s.set_tuning(vcycle_fused=2, vcycle_rhs_per_block=rpb, vcycle_tile=tile)
            y2 = to_np(s.apply("vcycle", f, l))
            for r in range(3):
                ref = lv.to_full(orc.vcycle(lv.to_unknowns(f[r]), l))
                assert rel(y2[r], ref) < tol, (l, rpb, tile, r, rel(y2[r], ref))
                assert rel(y2[r], y0[r]) < bound, (l, rpb, tile, r, rel(y2[r], y0[r]))
    s.close()


@pytest.mark.parametrize("prec,basis16", [("fp64", False), ("mixed_bf16", False),
                                          ("mixed_bf16", True), ("mixed", True)])
def test_staged_vcycle_solve_matches_fused(prec, basis16):
    """A batched solve whose right-hand sides converge at different
    iterations (so the staged kernels skip done RHS inside their groups)
    gives the same iterations (+-1) and solutions with the staged multi-RHS
    V-cycle as with the fused one.  With the FP16 inner basis the staged
    V-cycle reads its right-hand side straight from the basis (padded rows)
    instead of from an FP32 copy."""
    n, k = 65, 40.0
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    b = wl.point_sources(n, n, [(32, 32), (5, 60), (60, 5)])
    out = []
    for tune in (dict(vcycle_fused=1),
                 dict(vcycle_fused=2, vcycle_rhs_per_block=2, vcycle_tile=1)):
        s = solver(n, n, h, k2, "sommerfeld", prec=prec, nrhs=3, coarse_tol=1e-6,
                   coarse_maxit=300, inner_basis_fp16=basis16)
        s.set_tuning(**tune)
        x, info = s.solve(torch.from_numpy(b).cuda(), tol=1e-8)
        out.append((to_np(x), [(i.outer_iters, i.inner_iters_total) for i in info]))
        s.close()
    for r in range(3):
        assert abs(out[0][1][r][0] - out[1][1][r][0]) <= 1, (r, out[0][1], out[1][1])
        assert rel(out[1][0][r], out[0][0][r]) < 1e-6, r


@pytest.mark.parametrize("bc", BCS)
def test_vcycle_bf16_storage(bc):
    """BF16-storage smoother: level vectors rounded to 8-bit mantissas
    (relative 2^-9 per stored value), FP32 arithmetic; the V-cycle stays
    within 2e-2 of the FP64 oracle's."""
    k2 = rk2(NY, NX, 6)
    s = solver(NX, NY, H, k2, bc, z="ho", prec="mixed_bf16")
    orc = Oracle(NX, NY, H, k2, bc, z="ho", coarsest="direct")
    for l in (0, 1, orc.L):
        lv = orc.levels[l]
        f = wl.random_complex((1, lv.ny, lv.nx), 30 + l)
        y = to_np(s.apply("vcycle", f, l))[0]
        ref = lv.to_full(orc.vcycle(lv.to_unknowns(f[0]), l))
        assert rel(y, ref) < (2e-2 if l < orc.L else 1e-6), (l, rel(y, ref))


@pytest.mark.parametrize("prec,basis16", [("mixed", True), ("mixed_bf16", False),
                                          ("mixed_bf16", True)])
def test_reduced_storage_solves_reach_fp64_residual(prec, basis16):
    """FP16 inner Krylov basis and / or BF16 V-cycle storage inside FP64
    FGMRES: every RHS still reaches a true FP64 residual <= 1e-6 (checked
    with the oracle's A); the iteration counts stay near the FP32 ones."""
    n, k = 129, 80.0
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    nodes = [(64, 64), (30, 90)]
    b = wl.point_sources(n, n, nodes)
    ref = solver(n, n, h, k2, "sommerfeld", prec="mixed", nrhs=2,
                 coarse_tol=1e-1, coarse_maxit=300)
    _, iref = ref.solve(b, tol=1e-6)
    s = solver(n, n, h, k2, "sommerfeld", prec=prec, nrhs=2, coarse_tol=1e-1,
               coarse_maxit=300, inner_basis_fp16=basis16)
    x, info = s.solve(b, tol=1e-6)
    orc = Oracle(n, n, h, k2, "sommerfeld", z="ho", coarsest="direct")
    lv = orc.levels[0]
    xs = to_np(x)
    for r in range(2):
        bu = lv.to_unknowns(b[r])
        res = np.linalg.norm(bu - orc.A @ lv.to_unknowns(xs[r])) / np.linalg.norm(bu)
        assert res <= 1e-6 and info[r].status == "HZ_OK", (r, res)
        assert info[r].outer_iters <= iref[r].outer_iters + 2
        assert info[r].inner_iters_total <= 1.3 * iref[r].inner_iters_total + 10


@pytest.mark.parametrize("bc,z,e", [("sommerfeld", "ho", "galerkin"),
                                    ("dirichlet", "bilinear", "galerkin"),
                                    ("sommerfeld", "ho", "red_glk2")])
def test_coarse_solve_and_precond(bc, z, e):
    n = 65
    h = 1.0 / 64
    k2 = np.full((n, n), 30.0 ** 2)
    s = solver(n, n, h, k2, bc, z=z, e=e, coarse_tol=1e-12, coarse_maxit=600)
    orc = Oracle(n, n, h, k2, bc, z=z, e=e, coarsest="direct",
                 coarse_tol=1e-12, coarse_maxit=600)
    lc = orc.levels[1]
    v1 = wl.random_complex((1, lc.ny, lc.nx), 7)
    v2 = to_np(s.apply("coarse_solve", v1))[0]
    exact = lc.to_full(spla.spsolve(orc.E.tocsc(), lc.to_unknowns(v1[0])))
    assert rel(v2, exact) < 1e-9
    its = s.last_inner_iters(1)[0]
    orc.inner_log = []
    orc.coarse_solve(lc.to_unknowns(v1[0]))
    assert abs(its - orc.inner_log[0]) <= 1, (its, orc.inner_log)
    v = wl.random_complex((1, n, n), 8)
    z_gpu = to_np(s.apply("precond", v))[0]
    z_orc = orc.levels[0].to_full(orc.adef1(orc.levels[0].to_unknowns(v[0])))
    assert rel(z_gpu, z_orc) < 1e-8


def _solve_pair(n, k, bc, z, e, tol, ctol, prec="fp64", nodes=None):
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    nodes = nodes or [wl.centre_node(n, n)]
    b = wl.point_sources(n, n, nodes)
    s = solver(n, n, h, k2, bc, z=z, e=e, prec=prec, nrhs=len(nodes),
               coarse_tol=ctol, coarse_maxit=1500, outer_maxit=200)
    x, info = s.solve(b, tol=tol)
    orc = Oracle(n, n, h, k2, bc, z=z, e=e, coarse_tol=ctol,
                 coarse_maxit=1500)
    return orc, b, to_np(x), info


def test_config1_fp64_iterations_and_residual():
    """81 x 81, k = 50, Dirichlet, bilinear str-Glk, tol 1e-6, coarse 1e-6."""
    orc, b, x, info = _solve_pair(81, 50, "dirichlet", "bilinear", "galerkin",
                                  1e-6, 1e-6)
    xo, io = orc.solve(b[0], tol=1e-6)
    assert info[0].status == "HZ_OK"
    assert abs(info[0].outer_iters - io.outer_iters) <= 1
    lv = orc.levels[0]
    r = np.linalg.norm(lv.to_unknowns(b[0]) - orc.A @ lv.to_unknowns(x[0]))
    assert r / np.linalg.norm(lv.to_unknowns(b[0])) <= 1e-6
    assert info[0].relres <= 1e-6
    tot = info[0].inner_iters_total
    assert abs(tot - io.inner_total) <= max(3, 0.05 * io.inner_total), \
        (tot, io.inner_total)


@pytest.mark.parametrize("bc,z,e", [("sommerfeld", "ho", "galerkin"),
                                    ("sommerfeld", "ho", "red_glk2"),
                                    ("dirichlet", "ho", "red_o2"),
                                    ("sommerfeld", "bilinear", "red_glk1"),
                                    ("sommerfeld", "ho", "red_o4"),
                                    ("sommerfeld", "ho", "red_cmpo4"),
                                    ("dirichlet", "bilinear", "red_cmpo4"),
                                    ("sommerfeld", "ho", "red_o6"),
                                    ("sommerfeld", "ho", "red_9pt"),
                                    ("sommerfeld", None, "galerkin")])
def test_solve_parity_tight(bc, z, e):
    """At tight tolerances GPU and oracle solutions agree to 1e-8."""
    orc, b, x, info = _solve_pair(65, 30, bc, z, e, 1e-11, 1e-11)
    xo, io = orc.solve(b[0], tol=1e-11)
    assert rel(x[0], xo) < 1e-8
    assert abs(info[0].outer_iters - io.outer_iters) <= 1


def test_solve_with_stored_galerkin_stencil_matches_oracle():
    """The whole solve with stcl-op-Glk: same operator as str-Glk, so the
    tight solution matches the oracle's to 1e-8 and the outer count +-1."""
    n, k = 65, 30
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    b = wl.point_sources(n, n, [wl.centre_node(n, n)])
    s = solver(n, n, h, k2, "sommerfeld", z="ho", e="galerkin",
               coarse_tol=1e-11, coarse_maxit=1500, outer_maxit=200)
    s.set_tuning(galerkin_apply=1)
    x, info = s.solve(b, tol=1e-11)
    orc = Oracle(n, n, h, k2, "sommerfeld", z="ho", e="galerkin",
                 coarse_tol=1e-11, coarse_maxit=1500)
    xo, io = orc.solve(b[0], tol=1e-11)
    assert rel(to_np(x)[0], xo) < 1e-8
    assert abs(info[0].outer_iters - io.outer_iters) <= 1


@pytest.mark.parametrize("bc,z,e", [("sommerfeld", "ho", "galerkin"),
                                    ("dirichlet", "bilinear", "galerkin")])
def test_gcr_outer_matches_oracle(bc, z, e):
    """Flexible GCR as the outer iteration (Sec. 6.3): at tight tolerances
    the GPU and the oracle GCR give the same outer count (+-1) and
    solutions within 1e-8."""
    n, k = 65, 30
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    b = wl.point_sources(n, n, [wl.centre_node(n, n)])
    s = solver(n, n, h, k2, bc, z=z, e=e, coarse_tol=1e-11, coarse_maxit=1500,
               outer_maxit=200, outer="gcr")
    x, info = s.solve(b, tol=1e-11)
    orc = Oracle(n, n, h, k2, bc, z=z, e=e, coarse_tol=1e-11, coarse_maxit=1500)
    xo, io = orc.solve_gcr(b[0], tol=1e-11)
    assert info[0].status == "HZ_OK"
    assert abs(info[0].outer_iters - io.outer_iters) <= 1
    assert rel(to_np(x)[0], xo) < 1e-8


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_gcr_loose_coarse_tolerance_keeps_accuracy(prec):
    """Sec. 6.3: with the coarse solver at tolerance 0.1, GCR still reaches
    the outer tolerance (true residual <= 1e-6, by the oracle's A) in about
    as many outer iterations as flexible GMRES."""
    n, k = 129, 80
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    nodes = wl.centre_cluster(n, n, 3)
    b = wl.point_sources(n, n, nodes)
    out = {}
    for outer in ("gcr", "fgmres"):
        s = solver(n, n, h, k2, "sommerfeld", z="ho", e="galerkin", prec=prec,
                   nrhs=3, coarse_tol=1e-1, coarse_maxit=300, outer_maxit=100,
                   outer=outer)
        x, info = s.solve(b, tol=1e-6)
        out[outer] = (to_np(x), info)
    lv = ops.Level(n, n, h, k2, "sommerfeld")
    A = ops.five_point(lv)
    xg, ig = out["gcr"]
    for r in range(3):
        bu = lv.to_unknowns(b[r])
        res = np.linalg.norm(bu - A @ lv.to_unknowns(xg[r])) / np.linalg.norm(bu)
        assert ig[r].status == "HZ_OK" and res <= 1e-6, (r, res)
        assert abs(ig[r].outer_iters - out["fgmres"][1][r].outer_iters) <= 3


@pytest.mark.parametrize("bc,z", [("sommerfeld", "ho"), ("dirichlet", "bilinear")])
def test_tlkm_preconditioner_and_solve_match_oracle(bc, z):
    """The practical TLKM preconditioner (Sec. 3.2.2) applied once, and a
    tight FGMRES solve with it, against the oracle (1e-8; outer +-1)."""
    n, k = 65, 30
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    s = solver(n, n, h, k2, bc, z=z, coarse_tol=1e-12, coarse_maxit=800,
               outer_maxit=200, precond="tlkm")
    orc = Oracle(n, n, h, k2, bc, z=z, coarsest="direct", coarse_tol=1e-12,
                 coarse_maxit=800, precond="tlkm")
    v = wl.random_complex((1, n, n), 9)
    z_gpu = to_np(s.apply("precond", v))[0]
    z_orc = orc.levels[0].to_full(orc.tlkm(orc.levels[0].to_unknowns(v[0])))
    assert rel(z_gpu, z_orc) < 1e-8
    b = wl.point_sources(n, n, [wl.centre_node(n, n)])
    x, info = s.solve(b, tol=1e-11)
    orc2 = Oracle(n, n, h, k2, bc, z=z, coarse_tol=1e-11, coarse_maxit=800,
                  precond="tlkm")
    xo, io = orc2.solve(b[0], tol=1e-11)
    assert info[0].status == "HZ_OK"
    assert abs(info[0].outer_iters - io.outer_iters) <= 1
    assert rel(to_np(x)[0], xo) < 1e-8


@pytest.mark.parametrize("bc,z", [("sommerfeld", "ho"), ("dirichlet", "bilinear")])
def test_three_level_deflation_matches_oracle(bc, z):
    """Three-level deflation (the level-1 coarse system solved by flexible
    GMRES with A-DEF1 deflating to level 2, ReD-Glk2 there): one coarse
    solve and a tight whole solve against the oracle (1e-8; outer +-1), and
    the mixed-precision form reaches the FP64 residual target."""
    n, k = 33, 15
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), float(k) ** 2)
    s = solver(n, n, h, k2, bc, z=z, coarse_tol=1e-10, coarse_maxit=400,
               outer_maxit=200, deflation_levels=2)
    orc = Oracle(n, n, h, k2, bc, z=z, coarsest="direct", coarse_tol=1e-10,
                 coarse_maxit=400, deflation_levels=2)
    lc = orc.levels[1]
    v1 = wl.random_complex((1, lc.ny, lc.nx), 17)
    v2 = to_np(s.apply("coarse_solve", v1))[0]
    ref = lc.to_full(orc.coarse_solve(lc.to_unknowns(v1[0])))
    assert rel(v2, ref) < 1e-8
    b = wl.point_sources(n, n, [wl.centre_node(n, n)])
    x, info = s.solve(b, tol=1e-11)
    orc2 = Oracle(n, n, h, k2, bc, z=z, coarse_tol=1e-10, coarse_maxit=400,
                  deflation_levels=2)
    xo, io = orc2.solve(b[0], tol=1e-11)
    assert info[0].status == "HZ_OK"
    assert abs(info[0].outer_iters - io.outer_iters) <= 1
    assert rel(to_np(x)[0], xo) < 1e-8
    sm = solver(n, n, h, k2, bc, z=z, prec="mixed", coarse_tol=1e-2,
                coarse_maxit=200, outer_maxit=100, deflation_levels=2)
    xm, im = sm.solve(b, tol=1e-6)
    lv = orc2.levels[0]
    bu = lv.to_unknowns(b[0])
    res = np.linalg.norm(bu - orc2.A @ lv.to_unknowns(to_np(xm)[0])) / np.linalg.norm(bu)
    assert im[0].status == "HZ_OK" and res <= 1e-6


@pytest.mark.parametrize("depth", [2, 3, 4])
def test_multilevel_deflation_matches_oracle(depth):
    """Recursive A-DEF1 down to level D = depth (flexible GMRES with A-DEF1
    on every coarse system above D, ReD-Glk2 below level 1, V-cycle GMRES at
    D; every level to the coarse tolerance): one level-1 coarse solve and a
    tight whole solve against the oracle (1e-8; outer +-1), the whole solve
    issued as CUDA graphs (one WHILE node per level, nested) and kernel by
    kernel giving the same iterations and solution, and the mixed-precision
    form reaching the FP64 residual target."""
    n, k = 33, 12.0
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    kw = dict(coarse_tol=1e-1, coarse_maxit=6, deflation_levels=depth)
    s = solver(n, n, h, k2, "sommerfeld", z="ho", nrhs=2, outer_maxit=200, **kw)
    orc = Oracle(n, n, h, k2, "sommerfeld", z="ho", **kw)
    lc = orc.levels[1]
    v1 = wl.random_complex((1, lc.ny, lc.nx), 17 + depth)
    v2 = to_np(s.apply("coarse_solve", v1))[0]
    ref = lc.to_full(orc.coarse_solve(lc.to_unknowns(v1[0])))
    assert rel(v2, ref) < 1e-8
    b = wl.point_sources(n, n, [wl.centre_node(n, n), (3, 29)])
    x, info = s.solve(b, tol=1e-11)
    sg = solver(n, n, h, k2, "sommerfeld", z="ho", nrhs=2, outer_maxit=200,
                cuda_graph=False, **kw)
    xg, ig = sg.solve(b, tol=1e-11)
    for r in range(2):
        xo, io = orc.solve(b[r], tol=1e-11)
        assert info[r].status == "HZ_OK"
        assert abs(info[r].outer_iters - io.outer_iters) <= 1, (r, info[r], io.outer_iters)
        assert rel(to_np(x)[r], xo) < 1e-8
        assert (ig[r].outer_iters, ig[r].inner_iters_total) == \
            (info[r].outer_iters, info[r].inner_iters_total)
        assert rel(to_np(xg)[r], to_np(x)[r]) < 1e-13
    sm = solver(n, n, h, k2, "sommerfeld", z="ho", prec="mixed", nrhs=2,
                outer_maxit=200, **kw)
    xm, im = sm.solve(b, tol=1e-6)
    lv = orc.levels[0]
    for r in range(2):
        bu = lv.to_unknowns(b[r])
        res = np.linalg.norm(bu - orc.A @ lv.to_unknowns(to_np(xm)[r])) / np.linalg.norm(bu)
        assert im[r].status == "HZ_OK" and res <= 1e-6


def test_mixed_precision_reaches_fp64_residual():
    n, k = 129, 80
    orc, b, x, info = _solve_pair(n, k, "sommerfeld", "ho", "galerkin", 1e-6,
                                  1e-1, prec="mixed")
    lv = orc.levels[0]
    bu = lv.to_unknowns(b[0])
    r = np.linalg.norm(bu - orc.A @ lv.to_unknowns(x[0])) / np.linalg.norm(bu)
    assert r <= 1e-6 and info[0].status == "HZ_OK"
    xd = lv.to_full(spla.spsolve(orc.A.tocsc(), bu))
    # error against the exact discrete solution, stated per result
    err = rel(x[0], xd)
    assert err < 1e-3, err


def test_batched_equals_single_and_host_io():
    n = 65
    nodes = [(32, 32), (10, 50), (40, 5), (60, 60)]
    h = 1.0 / 64
    k2 = rk2(n, n, 9, 20, 40)
    b = wl.point_sources(n, n, nodes)
    sb = solver(n, n, h, k2, "sommerfeld", nrhs=4, coarse_tol=1e-6)
    xb, ib = sb.solve(b, tol=1e-8)
    s1 = solver(n, n, h, k2, "sommerfeld", nrhs=1, coarse_tol=1e-6)
    for r in range(4):
        x1, i1 = s1.solve(b[r:r + 1], tol=1e-8)
        assert i1[0].outer_iters == ib[r].outer_iters
        assert rel(to_np(xb[r]), to_np(x1[0])) < 1e-12
    bh = torch.from_numpy(b).pin_memory()
    xh, ih = sb.solve_host(bh, tol=1e-8)
    assert rel(xh.numpy(), to_np(xb)) < 1e-12


@pytest.mark.parametrize("bc,prec,basis16", [("sommerfeld", "fp64", False),
                                             ("dirichlet", "mixed", False),
                                             ("sommerfeld", "mixed_bf16", True)])
def test_cuda_graph_loop_equals_host_issued_loop(bc, prec, basis16):
    """The default path runs each outer iteration as one CUDA graph whose
    inner loop is a device-side WHILE node; with no_cuda_graph the same
    kernels are issued one by one.  Both must give the same iteration
    counts and the same solution (the kernels are deterministic), on two
    solves in a row (the second replays the cached graph), and the kernel
    counter must account for the kernels run inside the WHILE bodies."""
    from paper_2308_06152_gb300 import _lib
    lib = _lib.load_library()
    k2 = rk2(NY, NX, 5, lo=10.0, hi=40.0)
    b = wl.random_complex((2, NY, NX), 77)
    out = {}
    for graph in (True, False):
        s = solver(NX, NY, H, k2, bc, prec=prec, nrhs=2, coarse_tol=1e-3,
                   coarse_maxit=200, inner_basis_fp16=basis16,
                   cuda_graph=graph)
        runs = []
        for _ in range(2):
            torch.cuda.synchronize()
            n0 = lib.hz_kernel_launches()
            x, infos = s.solve(b, tol=1e-8)
            torch.cuda.synchronize()
            runs.append((to_np(x), infos, lib.hz_kernel_launches() - n0))
        s.close()
        out[graph] = runs
    for (xg, ig, ng), (xe, ie, ne) in zip(out[True], out[False]):
        for r in range(2):
            assert ig[r].status == ie[r].status == "HZ_OK"
            assert ig[r].outer_iters == ie[r].outer_iters
            assert ig[r].inner_iters_total == ie[r].inner_iters_total
            assert rel(xg[r], xe[r]) < 1e-13
        # the host-issued loop runs up to 3 extra (early-exit) inner steps
        # per coarse solve; the graph adds two small loop-control kernels
        assert 0.7 * ne < ng < 1.3 * ne, (ng, ne)
    assert rel(out[True][0][0], out[True][1][0]) == 0.0


@pytest.mark.parametrize("prec,basis16", [("fp64", False), ("mixed", True)])
def test_gram_schmidt_kernel_variants_agree(prec, basis16):
    """The register-pipelined and the two TMA-ring Gram-Schmidt kernels sum
    in different orders only: the same iteration counts (+-1) and solutions
    within rounding of each other (FP64 1e-9; mixed 1e-5, the FP32
    preconditioner's reach)."""
    k2 = rk2(NY, NX, 6, lo=10.0, hi=40.0)
    b = wl.random_complex((3, NY, NX), 78)
    res = {}
    for v in (0, 1, 2):
        s = solver(NX, NY, H, k2, "sommerfeld", prec=prec, nrhs=3,
                   coarse_tol=1e-3, coarse_maxit=200, inner_basis_fp16=basis16)
        s.set_tuning(mdot_kernel=v, maxpy_kernel=(v + 1) % 3)
        t = s.get_tuning()
        assert t["mdot_kernel"] == v and t["maxpy_kernel"] == (v + 1) % 3
        x, infos = s.solve(b, tol=1e-9)
        s.close()
        res[v] = (to_np(x), infos)
    tol = 1e-9 if prec == "fp64" else 1e-5
    x0, i0 = res[0]
    for v in (1, 2):
        xv, iv = res[v]
        for r in range(3):
            assert iv[r].status == "HZ_OK"
            assert abs(iv[r].outer_iters - i0[r].outer_iters) <= 1
            assert rel(xv[r], x0[r]) < tol, (v, r)


def test_autotune_picks_valid_choices_and_caches(tmp_path):
    """hz_autotune times every candidate, keeps the fastest of each, and a
    solve with the tuned choices still matches the default choices'; the
    JSON cache returns the same choice without timing."""
    k2 = rk2(NY, NX, 7, lo=10.0, hi=40.0)
    b = wl.random_complex((2, NY, NX), 79)
    s = solver(NX, NY, H, k2, "sommerfeld", prec="mixed", nrhs=2,
               coarse_tol=1e-3, coarse_maxit=100)
    x0, i0 = s.solve(b, tol=1e-8)
    cache = str(tmp_path / "tune.json")
    out = s.autotune(2, cache=cache)
    assert not out["cached"]
    ms = out["ms"]
    assert all(ms[c] > 0 for c in s.TUNE_CANDIDATES), ms
    t = out["tuning"]
    assert t == s.get_tuning()
    for cls in ("mdot_kernel", "maxpy_kernel"):
        assert t[cls] == min(range(3), key=lambda v: ms[f"{cls}={v}"])
    rpb = min((0, 8, 4), key=lambda v: ms[f"e_rhs_per_block={v}"])
    assert t["e_rhs_per_block"] == rpb
    pairs = 1 if ms["e_column_pairs=1"] < ms[f"e_rhs_per_block={rpb}"] else 0
    assert t["e_column_pairs"] == pairs
    assert ms["galerkin_apply=1"] == min(ms[f"e_rhs_per_block={rpb}"],
                                         ms["e_column_pairs=1"])
    ga = 1 if ms["galerkin_apply=1"] < ms["galerkin_apply=0"] else 0
    assert t["galerkin_apply"] == ga
    vc = [c for c in s.TUNE_CANDIDATES if c.startswith("vcycle_fused")]
    best = dict(kv.split("=") for kv in min(vc, key=lambda c: ms[c]).split(","))
    assert t["vcycle_fused"] == int(best["vcycle_fused"])
    if "rpb" in best:
        assert t["vcycle_rhs_per_block"] == int(best["rpb"])
        assert t["vcycle_tile"] == int(best["tile"])
    x1, i1 = s.solve(b, tol=1e-8)
    for r in range(2):
        assert i1[r].status == "HZ_OK"
        assert abs(i1[r].outer_iters - i0[r].outer_iters) <= 1
        assert rel(to_np(x1)[r], to_np(x0)[r]) < 1e-5
    s2 = solver(NX, NY, H, k2, "sommerfeld", prec="mixed", nrhs=2,
                coarse_tol=1e-3, coarse_maxit=100)
    again = s2.autotune(2, cache=cache)
    assert again["cached"] and again["tuning"] == t
    assert s2.get_tuning() == t


def test_group_of_uneven_grids_equals_separate_solves():
    """hz_solve_group on three grids of different shapes, boundary types and
    coarse operators, with different RHS counts: each member gets the same
    iteration counts and the same solution (the same kernels in the same
    order per member; FP64 to 1e-13) as its own separate solve."""
    from paper_2308_06152_gb300.api import solve_group
    specs = [(97, 73, 1.0 / 96, "sommerfeld", "ho", "galerkin", 2, 11),
             (65, 129, 1.0 / 64, "dirichlet", "bilinear", "galerkin", 1, 12),
             (129, 65, 1.0 / 128, "sommerfeld", "ho", "red_glk2", 3, 13)]
    for prec in ("fp64", "mixed"):
        solvers, bs = [], []
        for nx, ny, h, bc, z, e, nr, seed in specs:
            k2 = rk2(ny, nx, seed, lo=8.0, hi=30.0)
            solvers.append(solver(nx, ny, h, k2, bc, z=z, e=e, prec=prec,
                                  nrhs=nr, coarse_tol=1e-3, coarse_maxit=200,
                                  inner_basis_fp16=(prec == "mixed"),
                                  cuda_graph=False))
            bs.append(wl.random_complex((nr, ny, nx), seed + 100))
        out = solve_group(solvers, bs, tol=1e-8)
        for s, b, (xg, ig) in zip(solvers, bs, out):
            xs, is_ = s.solve(b, tol=1e-8)
            for r in range(b.shape[0]):
                assert ig[r].status == "HZ_OK"
                assert ig[r].outer_iters == is_[r].outer_iters
                assert ig[r].inner_iters_total == is_[r].inner_iters_total
                assert rel(to_np(xg)[r], to_np(xs)[r]) < 1e-13, (prec, r)
    # members must agree in precision class
    from paper_2308_06152_gb300.api import HzError
    a = solver(33, 33, 1 / 32, rk2(33, 33, 1), "sommerfeld", prec="fp64")
    c = solver(33, 33, 1 / 32, rk2(33, 33, 1), "sommerfeld", prec="mixed")
    with pytest.raises(HzError):
        solve_group([a, c], [wl.random_complex((1, 33, 33), 1)] * 2)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_group_graph_equals_eager_group(prec):
    """hz_solve_group issued as one CUDA graph per outer iteration (members'
    kernels on concurrent branches, the inner solves in a WHILE node) gives
    every member the iterations and solution of the same group issued
    kernel by kernel (1e-13), with far fewer host launch operations; the
    counts of both forms are printed."""
    from paper_2308_06152_gb300._lib import load_library
    from paper_2308_06152_gb300.api import solve_group
    lib = load_library()
    specs = [(97, 73, 1.0 / 96, "sommerfeld", "ho", "galerkin", 2, 11),
             (65, 129, 1.0 / 64, "dirichlet", "bilinear", "galerkin", 1, 12),
             (129, 65, 1.0 / 128, "sommerfeld", "ho", "red_glk2", 3, 13)]
    res, ops = {}, {}
    for graph in (False, True):
        solvers, bs = [], []
        for nx, ny, h, bc, z, e, nr, seed in specs:
            k2 = rk2(ny, nx, seed, lo=8.0, hi=30.0)
            solvers.append(solver(nx, ny, h, k2, bc, z=z, e=e, prec=prec, nrhs=nr,
                                  coarse_tol=1e-3, coarse_maxit=200,
                                  inner_basis_fp16=(prec == "mixed"), cuda_graph=graph))
            bs.append(wl.random_complex((nr, ny, nx), seed + 100))
        torch.cuda.synchronize()
        h0, k0 = lib.hz_host_launches(), lib.hz_kernel_launches()
        res[graph] = solve_group(solvers, bs, tol=1e-8)
        torch.cuda.synchronize()
        ops[graph] = (lib.hz_host_launches() - h0, lib.hz_kernel_launches() - k0)
    for (xe, ie), (xg, ig) in zip(res[False], res[True]):
        for r in range(len(ie)):
            assert ig[r].status == "HZ_OK"
            assert (ig[r].outer_iters, ig[r].inner_iters_total) == \
                (ie[r].outer_iters, ie[r].inner_iters_total)
            assert rel(to_np(xg)[r], to_np(xe)[r]) < 1e-13, (prec, r)
    print(f"group {prec}: host launches eager {ops[False][0]}, graphs {ops[True][0]}; "
          f"kernels {ops[False][1]} / {ops[True][1]}")
    # the graphs launch two loop-control kernels per inner iteration that the
    # host-issued form does not (the all-done flag, the WHILE condition)
    assert ops[True][0] * 5 < ops[False][0]


def test_timeout_path_with_fault_drill():
    """The TMA-ring dot kernel bounds every pipeline wait.  With the fault
    drill its producer warp issues no copies and the bound is 1 ms, so every
    consumer wait runs out with nothing in flight: the solve returns
    HZ_TIMEOUT instead of hanging.  After the drill is lifted the next solve
    on the same solver succeeds and gives the result of a solver that never
    saw the drill (the flag was cleared as it was reported)."""
    from paper_2308_06152_gb300._lib import load_library
    from paper_2308_06152_gb300.api import HzError
    lib = load_library()
    n, k = 65, 40.0
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    b = wl.point_sources(n, n, [(32, 32), (10, 50)])
    kw = dict(nrhs=2, coarse_tol=1e-6, coarse_maxit=300)
    ref = solver(n, n, h, k2, "sommerfeld", **kw)
    ref.set_tuning(mdot_kernel=1)
    x_ref, i_ref = ref.solve(b, tol=1e-8)
    s = solver(n, n, h, k2, "sommerfeld", **kw)
    s.set_tuning(mdot_kernel=1)
    assert lib.hz_fault_drill(None, 1, 1e-3) == 1
    assert lib.hz_fault_drill(s.handle, 1, 3.0) == 1
    assert lib.hz_fault_drill(s.handle, 1, 1e-3) == 0
    with pytest.raises(HzError) as err:
        s.solve(b, tol=1e-8)
    assert err.value.status == 7          # HZ_TIMEOUT
    assert lib.hz_fault_drill(s.handle, 0, 2.0) == 0
    x, info = s.solve(b, tol=1e-8)
    for r in range(2):
        assert info[r].status == "HZ_OK"
        assert info[r].outer_iters == i_ref[r].outer_iters
        assert rel(to_np(x)[r], to_np(x_ref)[r]) < 1e-13


@pytest.mark.parametrize("graph", [True, False])
def test_restarted_fgmres_matches_oracle(graph):
    """GMRES(m) as the outer iteration (hz_desc.restart = m): after every m
    iterations x is formed and the Arnoldi process starts again from
    b - A x with the stopping reference ||b|| kept.  The GPU matches the
    oracle's restarted flexible GMRES with the same m (outer iterations
    +-1, solution 1e-8), issued as graphs or kernel by kernel, and the
    restarted solve needs at least as many iterations as the full one."""
    n, k = 65, 40.0
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    b = wl.point_sources(n, n, [wl.centre_node(n, n), (5, 60)])
    kw = dict(nrhs=2, coarse_tol=1e-10, coarse_maxit=400, outer_maxit=200,
              cuda_graph=graph)
    s = solver(n, n, h, k2, "sommerfeld", restart=3, **kw)
    x, info = s.solve(b, tol=1e-10)
    full = solver(n, n, h, k2, "sommerfeld", **kw)
    xf, if_ = full.solve(b, tol=1e-10)
    orc = Oracle(n, n, h, k2, "sommerfeld", coarse_tol=1e-10, coarse_maxit=400)
    for r in range(2):
        xo, io = orc.solve(b[r], tol=1e-10, restart=3)
        assert info[r].status == "HZ_OK"
        assert abs(info[r].outer_iters - io.outer_iters) <= 1, (info[r], io.outer_iters)
        assert info[r].outer_iters >= if_[r].outer_iters
        assert rel(to_np(x)[r], xo) < 1e-8
        assert rel(to_np(x)[r], to_np(xf)[r]) < 1e-7


@pytest.mark.parametrize("levels", [1, 2])
def test_async_solve_matches_synchronous_solve(levels):
    """hz_solve_async enqueues the whole solve as one CUDA graph (the outer
    loop a device-side WHILE node holding the inner loop, and with
    three-level deflation the level-2 loop inside that) and returns at once;
    after the stream reaches its end, x and the device-side report equal
    hz_solve's (iterations, status, solution to 1e-13), on a first and a
    replayed call."""
    # (three-level deflation on a resolved coarse level: kh = 0.31 on the
    # fine grid, 1.25 on level 2)
    n, k = 65, (40.0 if levels == 1 else 20.0)
    h = 1.0 / (n - 1)
    k2 = np.full((n, n), k * k)
    b = torch.from_numpy(wl.point_sources(n, n, [(32, 32), (10, 50)])).cuda()
    kw = dict(nrhs=2, coarse_tol=1e-3 if levels > 1 else 1e-6,
              coarse_maxit=60 if levels > 1 else 300, outer_maxit=60,
              deflation_levels=levels)
    ref = solver(n, n, h, k2, "sommerfeld", **kw)
    x1, i1 = ref.solve(b, tol=1e-8)
    s = solver(n, n, h, k2, "sommerfeld", **kw)
    for call in range(2):
        x2, info = s.solve_async(b, tol=1e-8)
        torch.cuda.synchronize()
        i2 = s.infos_from_device(info)
        for r in range(2):
            assert i2[r].status == "HZ_OK"
            assert (i2[r].outer_iters, i2[r].inner_iters_total, i2[r].inner_iters_max) == \
                (i1[r].outer_iters, i1[r].inner_iters_total, i1[r].inner_iters_max)
            assert abs(i2[r].relres - i1[r].relres) <= 1e-12 * max(i1[r].relres, 1e-30)
            assert rel(to_np(x2)[r], to_np(x1)[r]) < 1e-13, (call, r)
    bad = solver(n, n, h, k2, "sommerfeld", restart=3, **kw)
    from paper_2308_06152_gb300.api import HzError
    with pytest.raises(HzError):
        bad.solve_async(b, tol=1e-8)


def test_gradient_group_equals_separate_gradients():
    """hz_gradient_group over two uneven grids (different shot counts,
    batches of 2 shots) equals each member's own hz_gradient (1e-12) and the
    oracle's sparse-LU gradient (1e-7)."""
    from paper_2308_06152_gb300.api import gradient_group
    cases = []
    # kh <= 0.8: the resolved regime of the method (an under-resolved
    # problem would need ~70 outer iterations per solve)
    for (nx, ny, h, omega, nsh, seed) in ((17, 13, 1 / 16, 10.0, 3, 31),
                                          (25, 33, 1 / 24, 14.0, 5, 32)):
        rng = np.random.default_rng(seed)
        m = rng.uniform(0.7, 1.3, size=(ny, nx))
        nodes = [(1 + (3 * s) % (nx - 2), 1 + s % 3) for s in range(nsh)]
        src = wl.point_sources(nx, ny, nodes)
        rec = wl.surface_receivers(nx, 0)
        d = (rng.standard_normal((nsh, nx))
             + 1j * rng.standard_normal((nsh, nx))) * 1e-3
        s = solver(nx, ny, h, omega ** 2 * m, "sommerfeld", z="ho", nrhs=2,
                   coarse_tol=1e-10, coarse_maxit=300)
        cases.append((s, omega, src, rec, d, m, nx, ny, h))
    import time
    t0 = time.perf_counter()
    out = gradient_group([c[0] for c in cases], [c[1] for c in cases],
                         [c[2] for c in cases], [c[3] for c in cases],
                         [c[4] for c in cases], tol=1e-11)
    t_group = time.perf_counter() - t0
    t_sep = 0.0
    for (s, omega, src, rec, d, m, nx, ny, h), (Jg, gg, ig) in zip(cases, out):
        t0 = time.perf_counter()
        J1, g1, _ = s.gradient(omega, src, rec, d, tol=1e-11)
        t_sep += time.perf_counter() - t0
        assert Jg == pytest.approx(J1, rel=1e-12)
        assert rel(to_np(gg), to_np(g1)) < 1e-12
        assert len(ig) == 2 * src.shape[0]
        assert all(i.status == "HZ_OK" for i in ig)
        J0, g0 = grd.misfit_and_gradient(nx, ny, h, m, omega, "sommerfeld", src,
                                         rec, d)
        assert Jg == pytest.approx(J0, rel=1e-8)
        assert rel(to_np(gg), g0) < 1e-7
    print(f"gradient group {t_group:.2f} s, separate {t_sep:.2f} s")


def test_edge_cases():
    from paper_2308_06152_gb300.api import Desc, HzError, Solver
    n = 33
    h = 1.0 / 32
    k2 = np.full((n, n), 400.0)
    s = solver(n, n, h, k2, "sommerfeld", nrhs=2, outer_maxit=3)
    b = np.zeros((2, n, n), complex)
    b[1, 16, 16] = 1.0
    x, info = s.solve(b, tol=1e-6)
    assert info[0].outer_iters == 0 and not np.any(to_np(x[0]))
    assert info[1].status in ("HZ_OK", "HZ_NOT_CONVERGED")
    # tolerance out of reach within outer_maxit
    x, info = s.solve(b[1:], tol=1e-15)
    assert info[0].status == "HZ_NOT_CONVERGED" and info[0].outer_iters == 3
    assert np.isfinite(info[0].relres)
    with pytest.raises(HzError):
        s.solve(np.zeros((3, n, n), complex))
    bn = b[1:].copy()
    bn[0, 3, 3] = np.nan
    x, info = s.solve(bn)
    assert info[0].status == "HZ_NAN"
    # smallest grids: one coarsening (5 x 5 -> 3 x 3) and none (3 x 3)
    s5 = solver(5, 5, 0.25, np.full((5, 5), 4.0), "sommerfeld", z="ho")
    o5 = Oracle(5, 5, 0.25, np.full((5, 5), 4.0), "sommerfeld", z="ho",
                coarse_tol=1e-12)
    b5 = wl.point_sources(5, 5, [(2, 2)])
    x5, i5 = s5.solve(b5, tol=1e-12)
    assert rel(to_np(x5[0]), o5.solve(b5[0], tol=1e-12)[0]) < 1e-9
    s3 = solver(3, 3, 0.5, np.full((3, 3), 1.0), "dirichlet", z=None)
    b3 = wl.point_sources(3, 3, [(1, 1)])
    x3, i3 = s3.solve(b3, tol=1e-12)
    assert abs(to_np(x3)[0, 1, 1] - 1.0 / (4 / 0.25 - 1.0)) < 1e-12
    with pytest.raises(HzError):
        Solver(Desc(34, 34, 1 / 33), np.ones((34, 34)))


def test_gradient_matches_oracle():
    nx, ny, h, omega = 17, 13, 1.0 / 16, 25.0
    rng = np.random.default_rng(11)
    m = rng.uniform(0.7, 1.3, size=(ny, nx))
    src = wl.point_sources(nx, ny, [(8, 6), (3, 2), (12, 9)])
    rec = wl.surface_receivers(nx, 0)
    d = (rng.standard_normal((3, nx)) + 1j * rng.standard_normal((3, nx))) * 1e-3
    s = solver(nx, ny, h, omega ** 2 * m, "sommerfeld", z="ho", nrhs=2,
               coarse_tol=1e-10, coarse_maxit=300)
    J, g, infos = s.gradient(omega, src, rec, d, tol=1e-12)
    J0, g0 = grd.misfit_and_gradient(nx, ny, h, m, omega, "sommerfeld", src,
                                     rec, d)
    assert J == pytest.approx(J0, rel=1e-8)
    assert rel(to_np(g), g0) < 1e-7
    assert len(infos) == 6 and all(i.status == "HZ_OK" for i in infos)


def test_autograd_gradient_matches_central_differences():
    """dJ/dm from the library's adjoint (through torch.autograd) against
    central differences of J computed by GPU forward solves (tol 1e-12),
    along random directions and single interior / edge / corner nodes."""
    from paper_2308_06152_gb300.api import Desc
    from paper_2308_06152_gb300.autograd import misfit
    nx, ny, h, omega = 17, 13, 1.0 / 16, 10.0
    rng = np.random.default_rng(21)
    m = torch.tensor(rng.uniform(0.7, 1.3, size=(ny, nx)), device="cuda",
                     requires_grad=True)
    src = wl.point_sources(nx, ny, [(8, 6), (3, 9)])
    rec = wl.surface_receivers(nx, 0)
    d = (rng.standard_normal((2, nx)) + 1j * rng.standard_normal((2, nx))) * 1e-3
    desc = Desc(nx, ny, h, bc="sommerfeld", z="ho", nrhs_max=2,
                coarse_tol=1e-10, coarse_maxit=300)
    J = misfit(m, desc, omega, src, rec, d, tol=1e-12)
    J.backward()
    g = m.grad.detach()
    dirs = [torch.tensor(rng.standard_normal((ny, nx)), device="cuda")
            for _ in range(3)]
    for (i, j) in ((8, 6), (0, 5), (0, 0)):
        e = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
        e[j, i] = 1.0
        dirs.append(e)
    with torch.no_grad():
        for dm in dirs:
            eps = 1e-4 * float(m.abs().max()) / float(dm.abs().max())
            jp = misfit(m + eps * dm, desc, omega, src, rec, d, tol=1e-12)
            jm = misfit(m - eps * dm, desc, omega, src, rec, d, tol=1e-12)
            fd = float(jp - jm) / (2 * eps)
            an = float((g * dm).sum())
            assert abs(fd - an) <= 1e-5 * abs(fd), (fd, an)


@pytest.mark.slow
def test_full_size_1281_mixed_batch_properties():
    """The bench workload (1281^2, k = 800, Sommerfeld, higher-order
    str-Glk, mixed precision, 16 shots): every RHS reaches a true FP64
    relative residual <= 1e-6 measured by the oracle's own A, and sampled
    entries of A x agree with the oracle."""
    model = wl.constant_k(1281, 800.0)
    nodes = wl.centre_cluster(1281, 1281, 16)
    b = wl.point_sources(1281, 1281, nodes)
    s = solver(1281, 1281, model.h, model.k2, "sommerfeld", z="ho",
               e="galerkin", prec="mixed", nrhs=16, coarse_tol=1e-1,
               coarse_maxit=200, outer_maxit=60)
    x, info = s.solve(b, tol=1e-6)
    lv = ops.Level(1281, 1281, model.h, model.k2, "sommerfeld")
    A = ops.five_point(lv)
    xs = to_np(x)
    for r in range(16):
        bu = lv.to_unknowns(b[r])
        res = np.linalg.norm(bu - A @ lv.to_unknowns(xs[r])) / np.linalg.norm(bu)
        assert res <= 1e-6 and info[r].status == "HZ_OK", (r, res)
    xr = wl.random_complex((1, 1281, 1281), 12)
    y = to_np(s.apply("helmholtz", xr))[0].reshape(-1)
    idx = np.random.default_rng(0).integers(0, 1281 * 1281, 4096)
    ref = (A @ lv.to_unknowns(xr[0]))[idx]
    np.testing.assert_allclose(y[idx], ref, rtol=1e-12,
                               atol=1e-12 * np.abs(ref).max())
