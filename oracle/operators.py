"""Assembled (CSR) operators of the method, FP64.  Test infrastructure only.

Grid conventions
----------------
A level is a vertex-centred grid of ``nx * ny`` nodes with spacing ``h``
(Sec. 2.1).  Arrays are ``(ny, nx)``, x fastest; the flat node index is
``j * nx + i``.  The coarse node ``(I, J)`` sits on the fine node
``(2I, 2J)`` (0-based form of the 1-based map ``(2i_c-1, 2j_c-1)``, Sec. 4).

Unknowns: every node under first-order Sommerfeld boundaries; the interior
nodes under homogeneous Dirichlet boundaries, where boundary nodes are fixed
at zero and interior rows drop their couplings to them (the Dirichlet rows
``ap = 1`` of Sec. 5.1 with zero boundary data give the same solution).

Coarsening (Sec. 4): a level is coarsened while both interval counts are
even and both coarse interval counts stay >= ``min_coarse_intervals``
(2 by default, the "at least 2 x 2 points" rule).  The wavenumber of a
coarse node is injected from the coincident fine node.
"""

import numpy as np
import scipy.sparse as sp

DIRICHLET = "dirichlet"
SOMMERFELD = "sommerfeld"


# --------------------------------------------------------------------------
# grid hierarchy
# --------------------------------------------------------------------------
def level_shapes(nx, ny, min_coarse_intervals=2):
    """Node counts of every level, finest first (Sec. 4 coarsening rule)."""
    shapes = [(nx, ny)]
    while True:
        cx, cy = shapes[-1]
        if (cx - 1) % 2 or (cy - 1) % 2:
            break
        ncx, ncy = (cx - 1) // 2 + 1, (cy - 1) // 2 + 1
        if ncx - 1 < min_coarse_intervals or ncy - 1 < min_coarse_intervals:
            break
        shapes.append((ncx, ncy))
    return shapes


class Level:
    """One grid level: shape, spacing, squared wavenumber and unknown set."""

    def __init__(self, nx, ny, h, k2, bc):
        if nx < 3 or ny < 3:
            raise ValueError("a level needs at least 3 x 3 nodes")
        if bc not in (DIRICHLET, SOMMERFELD):
            raise ValueError("bc must be 'dirichlet' or 'sommerfeld'")
        self.nx, self.ny, self.h, self.bc = int(nx), int(ny), float(h), bc
        self.k2 = np.asarray(k2, dtype=np.float64).reshape(ny, nx)
        mask = np.ones((ny, nx), dtype=bool)
        if bc == DIRICHLET:
            mask[0, :] = mask[-1, :] = False
            mask[:, 0] = mask[:, -1] = False
        self.mask = mask
        self.unk = np.flatnonzero(mask.ravel())
        self.n = self.unk.size

    def to_unknowns(self, u_full):
        return np.asarray(u_full, dtype=np.complex128).reshape(-1)[self.unk]

    def to_full(self, vec):
        out = np.zeros(self.nx * self.ny, dtype=np.complex128)
        out[self.unk] = vec
        return out.reshape(self.ny, self.nx)


def build_levels(nx, ny, h, k2, bc, min_coarse_intervals=2):
    """Levels 0..L with doubled spacing and injected wavenumber (Sec. 4)."""
    shapes = level_shapes(nx, ny, min_coarse_intervals)
    levels = [Level(nx, ny, h, k2, bc)]
    for (cx, cy) in shapes[1:]:
        prev = levels[-1]
        levels.append(Level(cx, cy, 2.0 * prev.h, prev.k2[::2, ::2], bc))
    return levels


def _restrict_to_unknowns(mat, rows_level, cols_level):
    return mat.tocsr()[rows_level.unk][:, cols_level.unk].tocsr()


# --------------------------------------------------------------------------
# Helmholtz and CSLP operators (Sec. 2.1, eqs. Helmstencil,
# Sommerfeldstencil1/2; Sec. 3.1 CSLP def; Sec. 5.1)
# --------------------------------------------------------------------------
def five_point_full(nx, ny, h, k2, bc, shift=1.0):
    """Full-grid (nx*ny square) 5-point operator -Lap_h - shift * k^2.

    Interior rows follow eq. (Helmstencil) with k^2 multiplied by ``shift``
    (``shift = 1`` gives A_h, ``shift = beta1 + i beta2`` gives the CSLP
    M_h of eq. (CSLP def)).  Under Sommerfeld boundaries the ghost node of
    eq. (GhostPoint) is eliminated: each boundary side of a node adds
    ``-2 i k h / h^2`` to the centre, removes the outward neighbour and
    doubles the opposite neighbour (eqs. Sommerfeldstencil1/2).  The
    boundary term uses the unshifted k for both A and M.
    """
    k2 = np.asarray(k2, dtype=np.float64).reshape(ny, nx)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    idx = jj * nx + ii
    inv_h2 = 1.0 / (h * h)
    diag = (4.0 * inv_h2 - shift * k2).astype(np.complex128)
    if bc == SOMMERFELD:
        nsides = ((ii == 0).astype(int) + (ii == nx - 1) + (jj == 0)
                  + (jj == ny - 1))
        diag = diag - 2j * nsides * np.sqrt(k2) / h
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [diag.ravel()]
    for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
        ni, nj = ii + di, jj + dj
        inside = (ni >= 0) & (ni < nx) & (nj >= 0) & (nj < ny)
        coef = np.full((ny, nx), -inv_h2, dtype=np.complex128)
        if bc == SOMMERFELD:
            mi, mj = ii - di, jj - dj
            mirror_out = ~((mi >= 0) & (mi < nx) & (mj >= 0) & (mj < ny))
            coef = np.where(mirror_out, 2.0 * coef, coef)
        rows.append(idx[inside])
        cols.append((nj * nx + ni)[inside])
        vals.append(coef[inside])
    n = nx * ny
    return sp.csr_matrix((np.concatenate(vals),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def five_point(level, shift=1.0):
    """A_h (shift=1) or M_h (shift=beta1+i*beta2) over the unknowns."""
    full = five_point_full(level.nx, level.ny, level.h, level.k2, level.bc,
                           shift)
    return _restrict_to_unknowns(full, level, level)


def symmetrizer(level):
    """Diagonal D with D*A symmetric: 1 interior, 1/2 edge, 1/4 corner
    under Sommerfeld boundaries (the ghost-eliminated rows carry the
    doubled -2/h^2 couplings); the identity under Dirichlet boundaries."""
    ny, nx = level.ny, level.nx
    d = np.ones((ny, nx))
    if level.bc == SOMMERFELD:
        d[0, :] *= 0.5
        d[-1, :] *= 0.5
        d[:, 0] *= 0.5
        d[:, -1] *= 0.5
    return d.reshape(-1)[level.unk]


# --------------------------------------------------------------------------
# transfer operators and deflation vectors (Sec. 3.2.1)
# --------------------------------------------------------------------------
def _p1_bilinear(nc):
    """1-D linear interpolation, eq. (linear iterpolation): a fine node on a
    coarse node copies it, a fine node between two averages them."""
    rows, cols, vals = [], [], []
    for I in range(nc):
        rows.append(2 * I); cols.append(I); vals.append(1.0)
        if I + 1 < nc:
            rows += [2 * I + 1, 2 * I + 1]
            cols += [I, I + 1]
            vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc - 1, nc))


def _p1_quadratic(nc):
    """1-D higher-order (quadratic Bezier) interpolation, eq. (quadratic
    approximation-a): a fine node on coarse node I takes
    (u_{I-1} + 6 u_I + u_{I+1}) / 8, a fine node between I and I+1 takes
    (u_I + u_{I+1}) / 2.  Coarse values outside the grid are zero."""
    rows, cols, vals = [], [], []
    for I in range(nc):
        for J, w in ((I - 1, 0.125), (I, 0.75), (I + 1, 0.125)):
            if 0 <= J < nc:
                rows.append(2 * I); cols.append(J); vals.append(w)
        if I + 1 < nc:
            rows += [2 * I + 1, 2 * I + 1]
            cols += [I, I + 1]
            vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * nc - 1, nc))


def prolongation(fine, coarse, kind="bilinear"):
    """Interpolation from ``coarse`` to ``fine`` over the unknowns.

    ``kind='bilinear'``: the tensor product of the 1-D linear rule, whose
    2-D stencil is (1/4)[1 2 1; 2 4 2; 1 2 1] (eq. bilinear operator).
    ``kind='ho'``: the tensor product of the 1-D quadratic rule, whose 2-D
    stencil is the (1/64) 5x5 stencil of eq. (higher-order intp-operator).
    """
    if kind == "bilinear":
        p1 = _p1_bilinear
    elif kind == "ho":
        p1 = _p1_quadratic
    else:
        raise ValueError(kind)
    assert fine.nx == 2 * coarse.nx - 1 and fine.ny == 2 * coarse.ny - 1
    full = sp.kron(p1(coarse.ny), p1(coarse.nx), format="csr")
    return _restrict_to_unknowns(full, fine, coarse)


def restriction(P):
    """R = Z^T / 4, the transpose scaled so that it is full weighting
    (eq. weight operator, stencil sum 1) for bilinear Z."""
    return (P.T / 4.0).tocsr()


# --------------------------------------------------------------------------
# coarse operators E (Sec. 5.2.1 - 5.2.4)
# --------------------------------------------------------------------------
# The 5x5 integer stencils printed for ReD-Glk: the Galerkin Laplacian
# (eq. Glk Laplace, scale 1/(256 (2h)^2)) and the constant-wavenumber
# mass term (eq. ReD-Glk Kh, scale k^2/64^2).  Rows are y offsets -2..2,
# columns x offsets -2..2 (both are symmetric).
GLK_LAPLACE = np.array([
    [-3, -44, -98, -44, -3],
    [-44, -112, 56, -112, -44],
    [-98, 56, 980, 56, -98],
    [-44, -112, 56, -112, -44],
    [-3, -44, -98, -44, -3]], dtype=np.float64)
GLK_MASS = np.array([
    [1, 28, 70, 28, 1],
    [28, 784, 1960, 784, 28],
    [70, 1960, 4900, 1960, 70],
    [28, 784, 1960, 784, 28],
    [1, 28, 70, 28, 1]], dtype=np.float64)


def galerkin(A0, Z):
    """str-Glk: E = R A_h Z with R = Z^T / 4, as an explicit sparse product
    of interpolation, fine operator and restriction (Sec. 5.2.1)."""
    return (restriction(Z) @ A0 @ Z).tocsr()


def red_o2(coarse):
    """ReD-O2: the 2nd-order Helmholtz stencil re-discretised on the coarse
    grid with the injected wavenumber (Sec. 5.2.3)."""
    return five_point(coarse, 1.0)


def _ghost_rule(bc, H, kb, u_bnd, u_in):
    """Ghost value outside a boundary node as a linear combination (dict
    node -> coefficient).  Sommerfeld: u_ghost = u_in + 2 i H k_b u_bnd
    (eq. GhostPoint); Dirichlet: u_ghost = 2 u_bnd - u_in
    (eq. DirchletGhostPoint)."""
    out = {}
    if bc == SOMMERFELD:
        for key, c in u_in.items():
            out[key] = out.get(key, 0) + c
        for key, c in u_bnd.items():
            out[key] = out.get(key, 0) + 2j * H * kb * c
    else:
        for key, c in u_bnd.items():
            out[key] = out.get(key, 0) + 2.0 * c
        for key, c in u_in.items():
            out[key] = out.get(key, 0) - c
    return out


def ghost_values(level):
    """Linear map from the real nodes to the values on the ring of ghost
    nodes one layer outside the grid, as dict (i, j) -> {node: coef}.

    Edge ghosts follow eq. (GhostPoint) (Sommerfeld) or eq.
    (DirchletGhostPoint) (Dirichlet) with k of the boundary node.  A corner
    ghost is reached by applying the rule once more along the ghost row (x
    first) or the ghost column (y first); the two orders are averaged.  In
    that second application the boundary node is itself a ghost; the
    boundary condition holds along the boundary line continued past the
    corner, so the rule takes the wavenumber of the corner node (the
    nearest real node on that line).  The wavenumber zero of a ghost node
    (Sec. 5.2.4) belongs to the mass stencil of eq. (ReD-Glk Kh), not to
    this rule: with zero here the corner ghost would lose one 2 i k H u
    term, an O(H) error that the 1/H^2 weight of the 5x5 Laplacian turns
    into an O(1/H) inconsistency of the corner rows.
    """
    nx, ny, H, bc = level.nx, level.ny, level.h, level.bc
    k = np.sqrt(level.k2)

    def real(i, j):
        return {j * nx + i: 1.0}

    def kb(i, j):
        if 0 <= i < nx and 0 <= j < ny:
            return k[j, i]
        return 0.0

    g = {}
    for j in range(ny):           # x ghosts on real rows
        g[(-1, j)] = _ghost_rule(bc, H, kb(0, j), real(0, j), real(1, j))
        g[(nx, j)] = _ghost_rule(bc, H, kb(nx - 1, j), real(nx - 1, j),
                                 real(nx - 2, j))
    for i in range(nx):           # y ghosts on real columns
        g[(i, -1)] = _ghost_rule(bc, H, kb(i, 0), real(i, 0), real(i, 1))
        g[(i, ny)] = _ghost_rule(bc, H, kb(i, ny - 1), real(i, ny - 1),
                                 real(i, ny - 2))
    for gi, bi, ii in ((-1, 0, 1), (nx, nx - 1, nx - 2)):
        for gj, bj, jj in ((-1, 0, 1), (ny, ny - 1, ny - 2)):
            # x rule on the ghost row gj, y rule on the ghost column gi,
            # both with k of the corner node (bi, bj)
            ox = _ghost_rule(bc, H, kb(bi, bj), g[(bi, gj)], g[(ii, gj)])
            oy = _ghost_rule(bc, H, kb(bi, bj), g[(gi, bj)], g[(gi, jj)])
            avg = {}
            for d in (ox, oy):
                for key, c in d.items():
                    avg[key] = avg.get(key, 0) + 0.5 * c
            g[(gi, gj)] = avg
    return g


def stencil_with_ghosts(level, rows_mask, coef_fn, radius, ghosts=None):
    """Assemble rows (full-grid) for nodes in ``rows_mask`` from a stencil of
    the given radius; neighbours one layer outside the grid are replaced by
    their ghost combination (``ghosts``, default ``ghost_values(level)``).
    ``coef_fn(i, j, di, dj, k2_nb)`` gives the coefficient of offset
    (di, dj), with k2_nb the squared wavenumber of that neighbour (zero at a
    ghost node)."""
    nx, ny = level.nx, level.ny
    g = ghost_values(level) if ghosts is None else ghosts
    rows, cols, vals = [], [], []
    for j in range(ny):
        for i in range(nx):
            if not rows_mask[j, i]:
                continue
            r = j * nx + i
            for dj in range(-radius, radius + 1):
                for di in range(-radius, radius + 1):
                    ni, nj = i + di, j + dj
                    inside = 0 <= ni < nx and 0 <= nj < ny
                    k2nb = level.k2[nj, ni] if inside else 0.0
                    c = coef_fn(i, j, di, dj, k2nb)
                    if c == 0:
                        continue
                    if inside:
                        rows.append(r); cols.append(nj * nx + ni)
                        vals.append(c)
                    else:
                        if (ni, nj) not in g:
                            raise ValueError("stencil reaches beyond the "
                                             "single ghost layer")
                        for col, w in g[(ni, nj)].items():
                            rows.append(r); cols.append(col)
                            vals.append(c * w)
    n = nx * ny
    return sp.csr_matrix((np.asarray(vals, dtype=np.complex128),
                          (rows, cols)), shape=(n, n))


def red_glk(coarse, variant=2, glk_scale=1.0):
    """ReD-Glk1 / ReD-Glk2 (Sec. 5.2.4).

    Interior coarse nodes use the Galerkin-derived 5x5 stencil
    [-Lap_2h] - [k^2_2h] of eqs. (Glk Laplace) and (ReD-Glk Kh), each entry
    of the mass part taking k^2 of its own coarse node, divided by 4 to
    match R = Z^T / 4.  Glk1: the two outermost rings of nodes use ReD-O2.
    Glk2: the outermost ring uses ReD-O2, the second ring the 5x5 stencil
    with ghost values (wavenumber zero at ghost nodes).  ``glk_scale``
    multiplies the 5x5 rows only: 4 gives the stencils as printed (the
    scale of Z^T A Z), for use with the unscaled restriction R = Z^T.
    """
    nx, ny, H = coarse.nx, coarse.ny, coarse.h
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    dist = np.minimum(np.minimum(ii, nx - 1 - ii), np.minimum(jj, ny - 1 - jj))
    o2_rows = dist <= (0 if variant == 2 else 1)
    lap = GLK_LAPLACE / (1024.0 * H * H)     # (1/4) (1/256) (1/H^2)
    mass = GLK_MASS / 16384.0                 # (1/4) (1/64^2)

    def coef(i, j, di, dj, k2nb):
        return lap[dj + 2, di + 2] - mass[dj + 2, di + 2] * k2nb

    full_glk = stencil_with_ghosts(coarse, ~o2_rows, coef, 2)
    full_o2 = five_point_full(nx, ny, H, coarse.k2, coarse.bc, 1.0)
    keep = sp.diags(o2_rows.ravel().astype(np.float64))
    full = (keep @ full_o2 + glk_scale * full_glk).tocsr()
    return _restrict_to_unknowns(full, coarse, coarse)


def _dist_to_boundary(nx, ny):
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return np.minimum(np.minimum(ii, nx - 1 - ii), np.minimum(jj, ny - 1 - jj))


def _red_cross(coarse, weights, ring):
    """Re-discretised operator: the 1-D second-difference weights
    ``weights`` (offsets -R..R, times 1/H^2) negated along x and y, minus
    k^2 of the node, on nodes at least ``ring`` nodes inside the grid; the
    others use the ReD-O2 row with its boundary rules."""
    nx, ny, H = coarse.nx, coarse.ny, coarse.h
    R = len(weights) // 2
    o2_rows = _dist_to_boundary(nx, ny) < ring
    w = -np.asarray(weights, dtype=np.float64) / (H * H)

    def coef(i, j, di, dj, k2nb):
        if di == 0 and dj == 0:
            return 2.0 * w[R] - k2nb
        if di != 0 and dj != 0:
            return 0.0
        return w[R + di + dj]

    full = stencil_with_ghosts(coarse, ~o2_rows, coef, R)
    full_o2 = five_point_full(nx, ny, H, coarse.k2, coarse.bc, 1.0)
    keep = sp.diags(o2_rows.ravel().astype(np.float64))
    return _restrict_to_unknowns((keep @ full_o2 + full).tocsr(), coarse, coarse)


def red_o6(coarse):
    """ReD-O6 (Sec. 5.2.3): the sixth-order second difference
    (2, -27, 270, -490, 270, -27, 2) / (180 H^2) along x and y minus k^2,
    on nodes whose 7-point cross stays inside the grid (at least 3 nodes
    from the boundary); the others use ReD-O2 (as for ReD-O4)."""
    return _red_cross(coarse, np.array([2, -27, 270, -490, 270, -27, 2]) / 180.0, 3)


def red_o4(coarse):
    """ReD-O4 (Sec. 5.2.3): coarse nodes whose 4th-order cross stays inside
    the grid use eq. (Helmstencil Oh4): the Laplacian
    [-1 16 -30 16 -1] / (12 H^2) along x and along y, minus k^2 of the node
    (the printed centre writes k^2 (2h)^2 inside the 1/(12 (2h)^2) factor,
    which would scale the wavenumber by 1/12; it is read as the plain -k^2
    of every other stencil of the paper).  Nodes within one node of the
    boundary, where the cross would leave the grid, use the ReD-O2 row with
    its boundary rules, as the paper does for its boundary points."""
    nx, ny, H = coarse.nx, coarse.ny, coarse.h
    o2_rows = _dist_to_boundary(nx, ny) <= 1
    s = 1.0 / (12.0 * H * H)
    side = {1: -16.0 * s, 2: 1.0 * s}

    def coef(i, j, di, dj, k2nb):
        if di == 0 and dj == 0:
            return 60.0 * s - k2nb
        if di != 0 and dj != 0:
            return 0.0
        return side[abs(di) + abs(dj)]

    full_o4 = stencil_with_ghosts(coarse, ~o2_rows, coef, 2)
    full_o2 = five_point_full(nx, ny, H, coarse.k2, coarse.bc, 1.0)
    keep = sp.diags(o2_rows.ravel().astype(np.float64))
    return _restrict_to_unknowns((keep @ full_o2 + full_o4).tocsr(), coarse, coarse)


# eq. (GeneralFormReD) with the Singer-Turkel coefficients (gamma = 1),
# Sec. 5.2.5: [A_2h] = [a] / H^2 - [b] k^2, rows y = -1..1, columns x.
def cmp_o4_weights(gamma=1.0):
    a0, a_s, a_c = 10.0 / 3.0, -2.0 / 3.0, -1.0 / 6.0
    b0 = 2.0 / 3.0 + gamma / 36.0
    b_s = 1.0 / 12.0 - gamma / 72.0
    b_c = gamma / 144.0
    a = np.array([[a_c, a_s, a_c], [a_s, a0, a_s], [a_c, a_s, a_c]])
    b = np.array([[b_c, b_s, b_c], [b_s, b0, b_s], [b_c, b_s, b_c]])
    return a, b


def ghost_values_cmp(level, fourth_order=True):
    """Ghost nodes one layer outside a Sommerfeld boundary for the compact
    3x3 schemes: ReD-cmpO4's 4th-order rule (Sec. 5.2.5)
    u_ghost = 2 i k H (1 - k^2 H^2 / 6) u_bnd + u_in, or (fourth_order
    False) the 2nd-order eq. (GhostPoint) u_ghost = 2 i k H u_bnd + u_in,
    with k of the boundary node; a corner ghost is the average of its two
    neighbouring edge ghosts."""
    nx, ny, H = level.nx, level.ny, level.h
    k = np.sqrt(level.k2)

    def rule(kb, b_node, in_node):
        corr = (1.0 - kb * kb * H * H / 6.0) if fourth_order else 1.0
        return {b_node: 2j * kb * H * corr, in_node: 1.0}

    g = {}
    for j in range(ny):
        g[(-1, j)] = rule(k[j, 0], j * nx, j * nx + 1)
        g[(nx, j)] = rule(k[j, nx - 1], j * nx + nx - 1, j * nx + nx - 2)
    for i in range(nx):
        g[(i, -1)] = rule(k[0, i], i, nx + i)
        g[(i, ny)] = rule(k[ny - 1, i], (ny - 1) * nx + i, (ny - 2) * nx + i)
    for gi, bi in ((-1, 0), (nx, nx - 1)):
        for gj, bj in ((-1, 0), (ny, ny - 1)):
            avg = {}
            for d in (g[(bi, gj)], g[(gi, bj)]):
                for key, c in d.items():
                    avg[key] = avg.get(key, 0) + 0.5 * c
            g[(gi, gj)] = avg
    return g


# ReD-9ptO2 (Appendix B): eq. (GeneralFormReD) with the coefficients the
# appendix fits at k = 80 (eq. optstcl_k80) and b0 = 1, b_s = b_c = 0.
def nine_point_o2_weights():
    a = np.array([[0.158, -1.316, 0.158], [-1.316, 4.632, -1.316],
                  [0.158, -1.316, 0.158]])
    b = np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 0.0]])
    return a, b


def red_9pt(coarse):
    """ReD-9ptO2 (Appendix B): [a] / H^2 - [b] k^2 with the appendix's
    coefficients; a second-order scheme, so Sommerfeld rows eliminate the
    ghost layer with eq. (GhostPoint), u_g = u_in + 2 i k H u_b (a corner
    ghost the average of its two neighbouring edge ghosts); Dirichlet rows
    only meet boundary nodes, which hold zero."""
    a, b = nine_point_o2_weights()
    ih2 = 1.0 / (coarse.h * coarse.h)

    def coef(i, j, di, dj, k2nb):
        return a[dj + 1, di + 1] * ih2 - b[dj + 1, di + 1] * k2nb

    ghosts = (ghost_values_cmp(coarse, fourth_order=False)
              if coarse.bc == SOMMERFELD else {})
    full = stencil_with_ghosts(coarse, coarse.mask, coef, 1, ghosts=ghosts)
    return _restrict_to_unknowns(full, coarse, coarse)


def red_cmpo4(coarse, gamma=1.0):
    """ReD-cmpO4 (Sec. 5.2.5): the compact 3x3 fourth-order stencil of
    eq. (GeneralFormReD), [a] / H^2 - [b] k^2, at every unknown.  Each entry
    of the mass part takes k^2 of its own node (zero at a ghost node, as for
    ReD-Glk); Sommerfeld boundary rows eliminate the ghost layer with
    ghost_values_cmp; Dirichlet rows only meet boundary nodes, which hold
    zero."""
    a, b = cmp_o4_weights(gamma)
    H = coarse.h
    ih2 = 1.0 / (H * H)

    def coef(i, j, di, dj, k2nb):
        return a[dj + 1, di + 1] * ih2 - b[dj + 1, di + 1] * k2nb

    ghosts = ghost_values_cmp(coarse) if coarse.bc == SOMMERFELD else {}
    full = stencil_with_ghosts(coarse, coarse.mask, coef, 1, ghosts=ghosts)
    return _restrict_to_unknowns(full, coarse, coarse)
