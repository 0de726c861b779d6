"""The heterogeneous-medium workloads at their full sizes, through the C ABI.

Wedge (three dipping layers, 600 x 1000 m) and the seeded layered-and-
faulted model (9200 x 3000 m) stand in for the paper's wedge and Marmousi
experiments (Sec. 6.2, 6.4); the gradient case follows the adjoint pattern
of the solver's gradient entry point.  At these sizes the oracle cannot
run the whole method, so each check uses what it can compute exactly:
- the oracle's assembled A gives the true residual of every solution;
- a sparse LU solve with that A gives the exact discrete solution, against
  which the error of each precision variant is stated and bounded;
- the oracle's sparse-LU adjoint gradient gives dJ/dm.
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


def solver(model, nrhs, **kw):
    from paper_2308_06152_gb300.api import Desc, Solver
    return Solver(Desc(model.nx, model.ny, model.h, bc="sommerfeld", z="ho",
                       e="galerkin", nrhs_max=nrhs, **kw), model.k2)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def true_residuals(A, lv, b, x):
    out = []
    for r in range(b.shape[0]):
        bu = lv.to_unknowns(b[r])
        out.append(np.linalg.norm(bu - A @ lv.to_unknowns(x[r]))
                   / np.linalg.norm(bu))
    return out


def test_wedge_small_matches_oracle_iterations():
    """Wedge at 10 Hz on 73 x 121 (kh = 0.35 at 1500 m/s), surface source
    at x = 300 m: the whole method on the oracle and on the GPU (FP64) give
    the same outer count (+-1) and solutions within 1e-7 at tol 1e-10."""
    m = wl.wedge(10.0, 73, 121)
    b = wl.point_sources(m.nx, m.ny, [((m.nx - 1) // 2, 0)])
    s = solver(m, 1, coarse_tol=1e-10, coarse_maxit=800, outer_maxit=200)
    x, info = s.solve(b, tol=1e-10)
    orc = Oracle(m.nx, m.ny, m.h, m.k2, "sommerfeld", z="ho", e="galerkin",
                 coarse_tol=1e-10, coarse_maxit=800)
    xo, io = orc.solve(b[0], tol=1e-10)
    assert info[0].status == "HZ_OK"
    assert abs(info[0].outer_iters - io.outer_iters) <= 1
    assert rel(x.cpu().numpy()[0], xo) < 1e-7


def test_wedge_40hz_precisions_against_exact_solution():
    """Wedge at 40 Hz on 289 x 481 (139,009 unknowns), coarse tolerance
    0.1: FP64, complex-FP32 and BF16-storage V-cycle (with an FP16 inner
    basis) preconditioners all reach a true FP64 residual <= 1e-6, and
    their errors against the exact discrete solution (sparse LU with the
    oracle's A) stay within a factor 2 of the FP64 preconditioner's."""
    m = wl.wedge(40.0, 289, 481)
    assert abs(m.kh_max() - 0.349) < 1e-3
    b = wl.point_sources(m.nx, m.ny, [((m.nx - 1) // 2, 0)])
    lv = ops.Level(m.nx, m.ny, m.h, m.k2, "sommerfeld")
    A = ops.five_point(lv)
    exact = lv.to_full(spla.spsolve(A.tocsc(), lv.to_unknowns(b[0])))
    errs = {}
    for prec, b16 in (("fp64", False), ("mixed", False), ("mixed_bf16", True)):
        s = solver(m, 1, prec=prec, inner_basis_fp16=b16, coarse_tol=1e-1,
                   coarse_maxit=300, outer_maxit=80)
        x, info = s.solve(b, tol=1e-6)
        xs = x.cpu().numpy()
        s.close()
        assert info[0].status == "HZ_OK", (prec, info[0])
        assert true_residuals(A, lv, b, xs)[0] <= 1e-6, prec
        errs[prec] = rel(xs[0], exact)
    # the discrete error at rel. residual 1e-6 (printed with -s)
    print("wedge 40 Hz error vs exact:", errs)
    assert errs["fp64"] < 1e-3
    for prec in ("mixed", "mixed_bf16"):
        assert errs[prec] < 2.0 * errs["fp64"] + 1e-6, errs


@pytest.mark.slow
def test_layered_faulted_64_shots_full_size():
    """The layered-and-faulted model at full size (2301 x 751 physical,
    padded to 2305 x 769, 1.77M nodes), 31.25 Hz, 64 surface shots in one
    batch, BF16-storage V-cycle with an FP16 inner basis in FP64 FGMRES:
    every shot reaches a true FP64 residual <= 1e-6 by the oracle's A."""
    m = wl.layered_faulted()
    assert (m.nx, m.ny) == (2305, 769) and m.physical == (2301, 751)
    nodes = wl.surface_line(m.physical[0] - 1, 64)
    b = wl.point_sources(m.nx, m.ny, nodes)
    s = solver(m, 64, prec="mixed_bf16", inner_basis_fp16=True,
               coarse_tol=1e-1, coarse_maxit=160, outer_maxit=30)
    x, info = s.solve(b, tol=1e-6)
    xs = x.cpu().numpy()
    s.close()
    del x
    torch.cuda.empty_cache()
    lv = ops.Level(m.nx, m.ny, m.h, m.k2, "sommerfeld")
    A = ops.five_point(lv)
    res = true_residuals(A, lv, b, xs)
    bad = [(r, res[r], info[r].status) for r in range(64)
           if not (res[r] <= 1e-6 and info[r].status == "HZ_OK")]
    assert not bad, bad[:5]


def _gradient_case(model, nshots, seed):
    """32 surface shots, receivers on every surface node, data from the
    model with +-5 % Gaussian velocity anomalies (computed by the oracle's
    sparse LU: the inverse crime is accepted), gradient at the background
    model."""
    omega = 2 * np.pi * model.freq
    m_true = wl.gaussian_anomalies(model, rel=0.05, seed=seed)
    m0 = model.k2 / omega ** 2
    step = max(1, (model.nx - 2) // nshots)
    nodes = [(1 + step * s, 0) for s in range(nshots)]
    src = wl.point_sources(model.nx, model.ny, nodes)
    rec = wl.surface_receivers(model.nx, 0)
    lv = ops.Level(model.nx, model.ny, model.h, omega ** 2 * m_true,
                   "sommerfeld")
    lu = spla.splu(ops.five_point(lv).tocsc())
    d = np.stack([lv.to_full(lu.solve(lv.to_unknowns(src[s]))).reshape(-1)[rec]
                  for s in range(nshots)])
    return omega, m0, src, rec, d


def test_gradient_uneven_grids_32_shots_each():
    """Config 5: the wedge (145 x 241, 20 Hz) and the reduced layered model
    (577 x 193, h = 16 m, 8 Hz) with 32 surface shots each, in one
    uneven-grid group (hz_gradient_group, batches of 16 shots): each
    model's dJ/dm matches the oracle's sparse-LU adjoint gradient."""
    from paper_2308_06152_gb300.api import Desc, Solver, gradient_group
    models = [wl.wedge(20.0, 145, 241),
              wl.layered_faulted(577, 193, h=16.0, freq=8.0, pad_to=None)]
    assert 0.5 < models[1].kh_max() < 0.55
    cases = [_gradient_case(m, 32, seed=1) for m in models]
    solvers = [Solver(Desc(m.nx, m.ny, m.h, bc="sommerfeld", z="ho",
                           e="galerkin", nrhs_max=16, coarse_tol=1e-3,
                           coarse_maxit=600, outer_maxit=300),
                      omega ** 2 * m0)
               for m, (omega, m0, src, rec, d) in zip(models, cases)]
    out = gradient_group(solvers, [c[0] for c in cases], [c[2] for c in cases],
                         [c[3] for c in cases], [c[4] for c in cases],
                         tol=1e-10)
    for m, (omega, m0, src, rec, d), (J, g, infos) in zip(models, cases, out):
        assert len(infos) == 64 and all(i.status == "HZ_OK" for i in infos)
        J0, g0 = grd.misfit_and_gradient(m.nx, m.ny, m.h, m0, omega,
                                         "sommerfeld", src, rec, d)
        assert J == pytest.approx(J0, rel=1e-7)
        assert rel(g.cpu().numpy(), g0) < 1e-6, m.name


def test_gradient_wedge_matches_central_differences():
    """dJ/dm on the 145 x 241 wedge (4 shots) against central differences
    of J along two random directions (1e-5 relative; solves to 1e-11)."""
    from paper_2308_06152_gb300.api import Desc, Solver
    model = wl.wedge(20.0, 145, 241)
    omega, m0, src, rec, d = _gradient_case(model, 4, seed=1)

    def make(m):
        return Solver(Desc(model.nx, model.ny, model.h, bc="sommerfeld", z="ho",
                           e="galerkin", nrhs_max=4, coarse_tol=1e-3,
                           coarse_maxit=600, outer_maxit=300),
                      omega ** 2 * m)

    s = make(m0)
    J, g, infos = s.gradient(omega, src, rec, d, tol=1e-11)
    s.close()
    assert all(i.status == "HZ_OK" for i in infos)
    g = g.cpu().numpy()
    rng = np.random.default_rng(5)
    for _ in range(2):
        dm = rng.standard_normal(m0.shape)
        eps = 1e-4 * np.abs(m0).max() / np.abs(dm).max()
        vals = []
        for sgn in (1.0, -1.0):
            sp_ = make(m0 + sgn * eps * dm)
            Jp, _, inf = sp_.gradient(omega, src, rec, d, tol=1e-11)
            sp_.close()
            assert all(i.status == "HZ_OK" for i in inf)
            vals.append(Jp)
        fd = (vals[0] - vals[1]) / (2 * eps)
        an = float((g * dm).sum())
        assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)
