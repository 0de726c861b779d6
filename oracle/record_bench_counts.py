"""Writes tests/golden/oracle_bench_counts.json: the oracle's own outer and
inner iteration counts and its wall time for one right-hand side of each
benchmark workload.  Calls only ``oracle/`` (and numpy for the inputs).

The counts scale the bounded CPU-baseline sample of ``bench.py`` (one outer
iteration timed live) to a whole solve.

    OPENBLAS_NUM_THREADS=1 python -m oracle.record_bench_counts [name ...]
"""

import json
import os
import sys
import time

import numpy as np

from oracle.solver import Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "tests", "golden", "oracle_bench_counts.json")

# name -> (n, k, bc, z, e, coarse_tol, coarse_maxit, tol): a unit point
# source at the centre of the unit square with constant wavenumber k.
WORKLOADS = {
    "mp2b_1281_k800": (1281, 800.0, "sommerfeld", "ho", "galerkin", 1e-1, 200,
                       1e-6),
    "mp2a_81_k50": (81, 50.0, "dirichlet", "bilinear", "galerkin", 1e-6, 3000,
                    1e-6),
}


def run(name):
    n, k, bc, z, e, ctol, cmax, tol = WORKLOADS[name]
    orc = Oracle(n, n, 1.0 / (n - 1), np.full((n, n), k * k), bc, z=z, e=e,
                 coarse_tol=ctol, coarse_maxit=cmax)
    b = np.zeros((n, n), complex)
    b[(n - 1) // 2, (n - 1) // 2] = 1.0
    t = time.time()
    _, info = orc.solve(b, tol=tol)
    return {"outer_iters": info.outer_iters,
            "inner_iters_total": info.inner_total,
            "relres": info.relres,
            "seconds": time.time() - t,
            "threads": os.environ.get("OPENBLAS_NUM_THREADS", "unset")}


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names or list(WORKLOADS):
        data[name] = run(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
