"""The method end to end, FP64 CPU: CSLP multigrid V-cycle, inner coarse
solve, A-DEF1 / APD preconditioner and outer flexible GMRES.  Test
infrastructure only.

Passages followed: CSLP and its V-cycle (Sec. 3.1, Sec. 5.1 last
paragraph, Sec. 6 coarsest-grid rule); deflation with Z = I_{2h}^h
(Sec. 3.2.1); A-DEF1 (Sec. 3.2.2, eq. ADEF1); the coarse problem
A_2h v_2 = v_1 solved by CSLP-preconditioned GMRES (Sec. 5.2, eqs.
matvec-restriction .. matvec-interpolation); flexible GMRES outer
iteration (Sec. 6.3).
"""

import numpy as np
import scipy.sparse.linalg as spla

from . import operators as ops
from .krylov import gcr_flexible, gmres_right, gmres_left


class SolveInfo:
    def __init__(self):
        self.outer_iters = 0
        self.inner_iters = []
        self.relres = np.nan
        self.converged = False

    @property
    def inner_total(self):
        return int(sum(self.inner_iters))


class Oracle:
    """Assembled hierarchy plus the method's steps.

    Parameters mirror the paper's defaults: beta = (1, -0.5) (Sec. 3.1),
    entering the CSLP through the coefficient printed in Sec. 5.1,
    Jacobi weight 0.8 with one pre- and one post-sweep (Sec. 3.1),
    coarsest-level GMRES to 1e-8 (Sec. 6), coarse tolerance 1e-6 (Sec. 6.3).

    ``z``: None (plain CSLP), 'bilinear' (A-DEF1) or 'ho' (APD).
    ``e``: 'galerkin' (str-Glk), 'red_o2', 'red_glk1', 'red_glk2',
    'red_o4', 'red_o6', 'red_cmpo4' or 'red_9pt'.
    ``coarsest``: 'gmres' (paper) or 'direct' (sparse LU; used where an
    exact coarsest solve is wanted for tight comparisons).
    ``precond``: 'adef1' (A-DEF1 / APD, eq. ADEF1) or 'tlkm' (the practical
    TLKM preconditioner of Sec. 3.2.2 with the coarse system of Sec. 5.2).
    ``deflation_levels``: D = 1 (the paper's two-level method) or D >= 2,
    multilevel deflation (the direction of Sec. 1 / Sec. 7): the coarse
    system of level l < D is solved by flexible GMRES preconditioned by
    A-DEF1 built from it, deflating to level l + 1 with ``e2`` there
    ('red_glk2' (default; Sec. 5.2.4 suggests ReD-Glk for multilevel use),
    'red_o2' or 'galerkin' = R_l E_l Z_l); the deepest system (level D) by
    V-cycle-preconditioned GMRES.  Every level uses the coarse tolerance.
    ``deflation_scaling``: 'consistent' (default) restricts with
    R_Z = Z^T / 4, under which R_Z A Z matches the re-discretised operators'
    scale (those of A_2h); 'printed' restricts with the unscaled R_Z = Z^T
    that the paper prints (the 1-D 1/2 [1 2 1] of Sec. 3.2.1 and the
    higher-order restriction of eq. O4 matrix-free restriction, stencil sums
    2 and 4), keeps the re-discretised operators and the ReD-O2 rows of
    ReD-Glk at the A_2h scale, and takes the 5x5 ReD-Glk rows as printed
    (the scale of Z^T A Z).  The Galerkin E and TLKM do not depend on the
    choice; the re-discretised E do.
    """

    def __init__(self, nx, ny, h, k2, bc, z="ho", e="galerkin",
                 beta=(1.0, -0.5), omega=0.8, min_coarse_intervals=2,
                 coarsest="gmres", coarsest_tol=1e-8, coarse_tol=1e-6,
                 coarse_maxit=3000, precond="adef1", deflation_levels=1,
                 e2="red_glk2", deflation_scaling="consistent"):
        self.levels = ops.build_levels(nx, ny, h, k2, bc,
                                       min_coarse_intervals)
        self.L = len(self.levels) - 1
        # CSLP coefficient as implemented in Sec. 5.1: ap = (4 - (beta1 -
        # beta2 i) k^2 h^2) / h^2, i.e. M = -Lap - (beta1 - i beta2) k^2.
        self.shift = complex(beta[0], -beta[1])
        self.omega = omega
        self.A = ops.five_point(self.levels[0], 1.0)
        self.M = [ops.five_point(lv, self.shift) for lv in self.levels]
        self.Dinv = [omega / m.diagonal() for m in self.M]
        self.P = [ops.prolongation(self.levels[l], self.levels[l + 1],
                                   "bilinear") for l in range(self.L)]
        self.R = [ops.restriction(p) for p in self.P]
        self.coarsest = coarsest
        self.coarsest_tol = coarsest_tol
        if coarsest == "direct":
            self._lu = spla.splu(self.M[self.L].tocsc())
        self.zkind, self.ekind = z, e
        if precond not in ("adef1", "tlkm") or (precond == "tlkm" and z is None):
            raise ValueError(precond)
        self.precond = self.adef1 if precond == "adef1" else self.tlkm
        self.coarse_tol, self.coarse_maxit = coarse_tol, coarse_maxit
        self.inner_log = []
        if deflation_scaling not in ("consistent", "printed") or (
                deflation_scaling == "printed" and deflation_levels != 1):
            raise ValueError("deflation_scaling must be 'consistent', or "
                             "'printed' with two levels")
        printed = deflation_scaling == "printed"
        glk_scale = 4.0 if printed else 1.0
        if z is not None:
            if self.L < 1:
                raise ValueError("deflation needs at least one coarsening")
            self.Z = ops.prolongation(self.levels[0], self.levels[1], z)
            self.RZ = self.Z.T.tocsr() if printed else ops.restriction(self.Z)
            if e == "galerkin":
                self.E = ((self.RZ @ self.A @ self.Z).tocsr() if printed
                          else ops.galerkin(self.A, self.Z))
            elif e == "red_o2":
                self.E = ops.red_o2(self.levels[1])
            elif e == "red_glk1":
                self.E = ops.red_glk(self.levels[1], 1, glk_scale)
            elif e == "red_glk2":
                self.E = ops.red_glk(self.levels[1], 2, glk_scale)
            elif e == "red_o4":
                self.E = ops.red_o4(self.levels[1])
            elif e == "red_cmpo4":
                self.E = ops.red_cmpo4(self.levels[1])
            elif e == "red_o6":
                self.E = ops.red_o6(self.levels[1])
            elif e == "red_9pt":
                self.E = ops.red_9pt(self.levels[1])
            else:
                raise ValueError(e)
        # multilevel deflation: coarse system l deflated again, down to D
        self.deflation_levels = deflation_levels
        if not isinstance(deflation_levels, (int, np.integer)) or deflation_levels < 1:
            raise ValueError("deflation_levels must be an integer >= 1")
        self.Zd, self.Rd, self.Ed = {}, {}, {}
        if deflation_levels >= 2:
            if z is None or self.L < deflation_levels or precond != "adef1":
                raise ValueError("multilevel deflation needs Z, A-DEF1 and "
                                 "deflation_levels coarsenings")
            self.Ed[1] = self.E
            for l in range(1, deflation_levels):
                lf, lc = self.levels[l], self.levels[l + 1]
                self.Zd[l] = ops.prolongation(lf, lc, z)
                self.Rd[l] = (self.Zd[l].T.tocsr() if printed
                              else ops.restriction(self.Zd[l]))
                if e2 == "galerkin":
                    self.Ed[l + 1] = (self.Rd[l] @ self.Ed[l] @ self.Zd[l]).tocsr()
                elif e2 == "red_glk2":
                    self.Ed[l + 1] = ops.red_glk(lc, 2, glk_scale)
                elif e2 == "red_o2":
                    self.Ed[l + 1] = ops.red_o2(lc)
                else:
                    raise ValueError(e2)
            # names of the three-level case
            self.Z1, self.R1, self.E2 = self.Zd[1], self.Rd[1], self.Ed[2]

    # ---- CSLP multigrid V-cycle (Sec. 3.1) -------------------------------
    def coarsest_solve(self, f):
        if self.coarsest == "direct":
            return self._lu.solve(f)
        ML = self.M[self.L]
        return gmres_right(lambda v: ML @ v, f, self.coarsest_tol,
                           maxit=max(ML.shape[0], 1)).x

    def vcycle(self, f, level=0):
        """One V-cycle for M_level x = f from x = 0: damped-Jacobi pre-sweep,
        full-weighting restriction of the residual, recursion, bilinear
        interpolation of the correction, damped-Jacobi post-sweep."""
        if level == self.L:
            return self.coarsest_solve(f)
        M, Dinv = self.M[level], self.Dinv[level]
        x = Dinv * f
        r = f - M @ x
        xc = self.vcycle(self.R[level] @ r, level + 1)
        x = x + self.P[level] @ xc
        x = x + Dinv * (f - M @ x)
        return x

    # ---- deflation (Sec. 3.2, 5.2) ----------------------------------------
    def coarse_solve(self, v1, tol=None, maxit=None):
        """E v2 = v1 by GMRES right-preconditioned with the V-cycle on the
        coarse CSLP (levels 1..L), x0 = 0.  With multilevel deflation the
        preconditioner is A-DEF1 of the coarse system itself (adef1_at),
        which contains an inexact solve, so the GMRES is flexible."""
        tol = self.coarse_tol if tol is None else tol
        maxit = self.coarse_maxit if maxit is None else maxit
        if self.deflation_levels >= 2:
            res = gmres_right(lambda v: self.E @ v, v1, tol, maxit,
                              prec=lambda v: self.adef1_at(1, v), flexible=True)
        else:
            res = gmres_right(lambda v: self.E @ v, v1, tol, maxit,
                              prec=lambda v: self.vcycle(v, 1))
        self.inner_log.append(res.iters)
        return res.x

    def solve_level(self, l, v):
        """E_l x = v (2 <= l <= D) to the coarse tolerance, x0 = 0: at the
        deepest level D by GMRES right-preconditioned with the V-cycle from
        level D, above it by flexible GMRES preconditioned by A-DEF1 of
        level l."""
        E = self.Ed[l]
        if l == self.deflation_levels:
            return gmres_right(lambda u: E @ u, v, self.coarse_tol,
                               self.coarse_maxit,
                               prec=lambda u: self.vcycle(u, l)).x
        return gmres_right(lambda u: E @ u, v, self.coarse_tol,
                           self.coarse_maxit, prec=lambda u: self.adef1_at(l, u),
                           flexible=True).x

    def adef1_at(self, l, v):
        """A-DEF1 for the coarse system of level l < D (eq. ADEF1 applied
        l levels down): M_l^-1 (v - E_l q) + q with q = Z_l E_{l+1}^-1 R_l v."""
        q = self.Zd[l] @ self.solve_level(l + 1, self.Rd[l] @ v)
        return self.vcycle(v - self.Ed[l] @ q, l) + q

    def coarse_solve_level2(self, v):
        """E_2 v2 = v (three-level deflation's level 2)."""
        return self.solve_level(2, v)

    def adef1_level1(self, v):
        """A-DEF1 for the level-1 coarse system E (three-level naming)."""
        return self.adef1_at(1, v)

    def deflation_Q(self, v):
        """Q v = Z E^{-1} R v with the inexact coarse solve (Sec. 5.2)."""
        return self.Z @ self.coarse_solve(self.RZ @ v)

    def adef1(self, v):
        """P_A-DEF1 v = M^{-1}(v - A Q v) + Q v (eq. ADEF1); without
        deflation vectors this is the plain CSLP V-cycle."""
        if self.zkind is None:
            return self.vcycle(v, 0)
        q = self.deflation_Q(v)
        return self.vcycle(v - self.A @ q, 0) + q

    def coarse_solve_tlkm(self, v1, tol=None, maxit=None):
        """The practical TLKM coarse system (Sec. 5.2, eq. TLKM CGP):
        I_h^2h I_2h^h M_2h^-1 A_2h v2 = v1 with I_h^2h I_2h^h = R_Z Z, M_2h^-1
        one V-cycle on the coarse CSLP from level 1 and A_2h = E, by GMRES on
        that operator (it already carries M_2h^-1), x0 = 0."""
        tol = self.coarse_tol if tol is None else tol
        maxit = self.coarse_maxit if maxit is None else maxit
        RZZ = self.RZ @ self.Z
        res = gmres_right(lambda v: RZZ @ self.vcycle(self.E @ v, 1), v1, tol,
                          maxit)
        self.inner_log.append(res.iters)
        return res.x

    def tlkm(self, v, gamma=1.0):
        """Practical TLKM preconditioner (Sec. 3.2.2):
        P v = (I - A~ Q~ + gamma Q~) M^-1 v with A~ = M^-1 A and
        Q~ = Z A~_2h^-1 R_Z, A~_2h replaced by the practical coarse operator
        of coarse_solve_tlkm; gamma = 1."""
        w = self.vcycle(v, 0)
        q = self.Z @ self.coarse_solve_tlkm(self.RZ @ w)
        return w - self.vcycle(self.A @ q, 0) + gamma * q

    # ---- outer solve (Sec. 6.3) -------------------------------------------
    def solve(self, b_full, tol=1e-6, maxit=500, x0_full=None, restart=None):
        """Flexible GMRES on A x = b right-preconditioned by A-DEF1 (restarted
        every ``restart`` iterations if given).  Returns the full-grid
        solution and a SolveInfo with the true relative residual."""
        lv = self.levels[0]
        b = lv.to_unknowns(b_full)
        x0 = None if x0_full is None else lv.to_unknowns(x0_full)
        self.inner_log = []
        res = gmres_right(lambda v: self.A @ v, b, tol, maxit, x0=x0,
                          prec=self.precond, flexible=True, restart=restart)
        info = SolveInfo()
        info.outer_iters = res.iters
        info.inner_iters = list(self.inner_log)
        bn = np.linalg.norm(b)
        info.relres = (np.linalg.norm(b - self.A @ res.x) / bn) if bn else 0.0
        info.converged = res.converged
        return lv.to_full(res.x), info

    def solve_gcr(self, b_full, tol=1e-6, maxit=500):
        """Flexible GCR on A x = b right-preconditioned by A-DEF1 (the
        outer iteration of Sec. 6.3).  Returns the full-grid solution and a
        SolveInfo with the true relative residual."""
        lv = self.levels[0]
        b = lv.to_unknowns(b_full)
        self.inner_log = []
        res = gcr_flexible(lambda v: self.A @ v, b, tol, maxit, prec=self.precond)
        info = SolveInfo()
        info.outer_iters = res.iters
        info.inner_iters = list(self.inner_log)
        bn = np.linalg.norm(b)
        info.relres = (np.linalg.norm(b - self.A @ res.x) / bn) if bn else 0.0
        info.converged = res.converged
        return lv.to_full(res.x), info

    def solve_left(self, b_full, tol=1e-6, maxit=500):
        """Algorithm 1 (left preconditioning, preconditioned residual), for
        comparison with the paper's iteration tables."""
        lv = self.levels[0]
        b = lv.to_unknowns(b_full)
        self.inner_log = []
        res = gmres_left(lambda v: self.A @ v, self.adef1, b, tol, maxit)
        info = SolveInfo()
        info.outer_iters = res.iters
        info.inner_iters = list(self.inner_log)
        bn = np.linalg.norm(b)
        info.relres = np.linalg.norm(b - self.A @ res.x) / bn
        info.converged = res.converged
        return lv.to_full(res.x), info

    # ---- full-grid wrappers used by the parity tests ----------------------
    def apply_full(self, mat, level, u_full):
        lv = self.levels[level]
        return lv.to_full(mat @ lv.to_unknowns(u_full))
