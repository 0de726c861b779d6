"""Prints the oracle's outer iteration counts beside those the paper prints
in Tables 2, 3 and 5 (Sec. 6.2), under both deflation-restriction scalings
of the oracle: the consistent R_Z = Z^T / 4 and the printed R_Z = Z^T.
Calls only ``oracle/``; the printed numbers come from the fixtures under
``tests/golden/`` (each with its citation).

    OPENBLAS_NUM_THREADS=1 python -m oracle.paper_tables

Every run is MP-2a (Dirichlet) or MP-2b (Sommerfeld): the unit square,
constant k, a unit point source at the centre, left-preconditioned GMRES
(Algorithm 1) to 1e-6, the coarse problem solved by CSLP-GMRES to 1e-6.
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


def outer(n, k, bc, z, e, precond, scaling):
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), k * k), bc, z=z, e=e,
                 coarse_tol=1e-6, precond=precond, deflation_scaling=scaling)
    b = np.zeros((n, n), complex)
    b[n // 2, n // 2] = 1.0
    bu = orc.levels[0].to_unknowns(b)
    return gmres_left(lambda v: orc.A @ v, orc.precond, bu, 1e-6, 300).iters


def row(label, cases, paper):
    res = {s: [outer(*c, s) for c in cases] for s in ("consistent", "printed")}
    fmt = lambda v: "/".join("-" if x is None else str(int(x)) for x in v)  # noqa: E731
    print(f"{label:34s} paper {fmt(paper):22s} Z^T/4 {fmt(res['consistent']):22s} "
          f"Z^T {fmt(res['printed'])}", flush=True)


def main():
    low = [("galerkin", "adef1"), ("red_o2", "adef1"), ("red_o2", "tlkm")]
    t23 = load("outer_counts_tables_2_3.txt")
    for table, bc in (("table2", ops.DIRICHLET), ("table3", ops.SOMMERFELD)):
        for r in t23[table]:
            n, k = int(r[0]), r[1]
            row(f"{table} {n}^2 k={k:g} Glk/O2/TLKM", [(n, k, bc, "bilinear", e, p)
                                                     for e, p in low], r[2:])
    t5 = load("table5_mp2b.txt")["outer"]
    for r in t5:
        n, k = int(r[0]), r[1]
        cols = [e for e, p in zip(E_COLS, r[2:]) if p is not None]
        row(f"table5 {n}^2 k={k:g} " + "/".join(c.replace("red_", "") for c in cols),
            [(n, k, ops.SOMMERFELD, "ho", e, "adef1") for e in cols],
            [p for p in r[2:] if p is not None])


if __name__ == "__main__":
    sys.exit(main())
