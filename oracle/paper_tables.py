"""Prints the oracle's outer iteration counts beside those the paper prints
in Tables 2, 3 and 5 (Sec. 6.2), under both deflation-restriction scalings
of the oracle: the consistent R_Z = Z^T / 4 and the printed R_Z = Z^T.
Calls only ``oracle/``; the printed numbers come from the fixtures under
``tests/golden/`` (each with its citation).

    OPENBLAS_NUM_THREADS=1 python -m oracle.paper_tables

Every run is MP-2a (Dirichlet) or MP-2b (Sommerfeld): the unit square,
constant k, a unit point source at the centre, left-preconditioned GMRES
(Algorithm 1) to 1e-6, the coarse problem solved by CSLP-GMRES.  Tables 2
and 3 run with a coarse tolerance of 1e-6; Table 5 with 1e-12, the
coarse-grid solver's tolerance that the introduction of Sec. 6 states for
the convergence study, and its lines add the mean inner iterations per
coarse solve beside the printed ones (in parentheses).
"""

import os
import sys

import numpy as np

from oracle import operators as ops
from oracle.krylov import gmres_left
from oracle.solver import Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")
E_COLS = ["galerkin", "red_o2", "red_o4", "red_cmpo4", "red_o6", "red_glk1",
          "red_glk2"]


def load(name):
    """'[key]' blocks of number rows ('C' = not run), '#' comments."""
    out, key = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                key = line[1:-1]
                out[key] = []
                continue
            out[key].append([None if t == "C" else float(t) for t in line.split()])
    return out


def counts(n, k, bc, z, e, precond, scaling, tau_c):
    """Outer iterations and mean inner iterations per coarse solve."""
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), k * k), bc, z=z, e=e,
                 coarse_tol=tau_c, precond=precond, deflation_scaling=scaling)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    bu = orc.levels[0].to_unknowns(b)
    orc.inner_log = []
    it = gmres_left(lambda v: orc.A @ v, orc.precond, bu, 1e-6, 300).iters
    return it, (float(np.mean(orc.inner_log)) if orc.inner_log else None)


def row(label, cases, paper, tau_c=1e-6, paper_inner=None):
    res = {s: [counts(*c, s, tau_c) for c in cases]
           for s in ("consistent", "printed")}

    def fmt(v, inner=None):
        out = []
        for i, x in enumerate(v):
            o = x[0] if isinstance(x, tuple) else x
            t = "-" if o is None else str(int(o))
            if inner is not None and inner[i] is not None:
                t += f"({int(round(inner[i]))})"
            out.append(t)
        return "/".join(out)

    show_inner = paper_inner is not None
    print(f"{label:34s} paper {fmt(paper, paper_inner):40s} "
          f"Z^T/4 {fmt(res['consistent'], [r[1] for r in res['consistent']] if show_inner else None):40s} "
          f"Z^T {fmt(res['printed'], [r[1] for r in res['printed']] if show_inner else None)}",
          flush=True)


def main():
    low = [("galerkin", "adef1"), ("red_o2", "adef1"), ("red_o2", "tlkm")]
    t23 = load("outer_counts_tables_2_3.txt")
    for table, bc in (("table2", ops.DIRICHLET), ("table3", ops.SOMMERFELD)):
        for r in t23[table]:
            n, k = int(r[0]), r[1]
            row(f"{table} {n}^2 k={k:g} Glk/O2/TLKM", [(n, k, bc, "bilinear", e, p)
                                                     for e, p in low], r[2:])
    t5 = load("table5_mp2b.txt")
    for r, ri in zip(t5["outer"], t5["inner"]):
        n, k = int(r[0]), r[1]
        cols = [e for e, p in zip(E_COLS, r[2:]) if p is not None]
        row(f"table5 {n}^2 k={k:g} " + "/".join(c.replace("red_", "") for c in cols),
            [(n, k, ops.SOMMERFELD, "ho", e, "adef1") for e in cols],
            [p for p in r[2:] if p is not None], tau_c=1e-12,
            paper_inner=[p for p in ri[2:] if p is not None])


if __name__ == "__main__":
    sys.exit(main())
