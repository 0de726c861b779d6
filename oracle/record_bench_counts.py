"""Writes tests/golden/oracle_bench_counts.json: for one right-hand side of
each benchmark workload, the oracle's own outer and inner iteration counts,
the wall time of its whole solve and the wall time of a bounded sample (the
calibration sample below) timed in the same process.  Calls only
``oracle/`` (and the seeded input generators for the inputs).

``bench.py`` times the same calibration sample on the host it runs on and
scales the recorded whole-solve time by the ratio of the two sample times,
so its CPU baseline is a timed whole solve of the oracle carried over to
that host's speed, not an extrapolation from iteration counts.

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

# inner iterations of the calibration sample (enough for about 10-30 s of
# work at the benchmark sizes)
SAMPLE_INNER = {"mp2b_1281_k800": 60, "layered_2305x769_b64": 60,
                "mp2a_81_k50": 400}


def workload(name):
    """(model, rhs full grid, bc, z, e, coarse_tol, coarse_maxit, tol) of one
    right-hand side of a benchmark workload: the first shot of its batch."""
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    from paper_2308_06152_gb300 import workloads as wl
    if name == "mp2b_1281_k800":
        m = wl.constant_k(1281, 800.0)
        b = wl.point_sources(m.nx, m.ny, [wl.centre_node(m.nx, m.ny)])[0]
        return m, b, "sommerfeld", "ho", "galerkin", 1e-1, 200, 1e-6
    if name == "mp2a_81_k50":
        m = wl.constant_k(81, 50.0)
        b = wl.point_sources(m.nx, m.ny, [wl.centre_node(m.nx, m.ny)])[0]
        return m, b, "dirichlet", "bilinear", "galerkin", 1e-6, 3000, 1e-6
    if name == "layered_2305x769_b64":
        m = wl.layered_faulted(2301, 751, freq=31.25)
        node = wl.surface_line(m.physical[0] - 1, 64)[0]
        b = wl.point_sources(m.nx, m.ny, [node])[0]
        return m, b, "sommerfeld", "ho", "galerkin", 1e-1, 160, 1e-6
    raise KeyError(name)


def make_oracle(name):
    m, b, bc, z, e, ctol, cmax, tol = workload(name)
    orc = Oracle(m.nx, m.ny, m.h, m.k2, bc, z=z, e=e, coarse_tol=ctol,
                 coarse_maxit=cmax)
    return orc, b, tol


def calibration_sample(orc, b, inner):
    """The first coarse solve of the first outer iteration of the oracle's
    solve (R_Z applied to the normalised right-hand side, then its
    CSLP-preconditioned GMRES), stopped after ``inner`` iterations.
    Returns its wall time in seconds."""
    lv = orc.levels[0]
    bu = lv.to_unknowns(b)
    v1 = orc.RZ @ (bu / np.linalg.norm(bu))
    t = time.perf_counter()
    orc.coarse_solve(v1, tol=1e-300, maxit=inner)
    return time.perf_counter() - t


def run(name):
    orc, b, tol = make_oracle(name)
    ts = calibration_sample(orc, b, SAMPLE_INNER[name])
    t = time.perf_counter()
    _, info = orc.solve(b, tol=tol)
    return {"outer_iters": info.outer_iters,
            "inner_iters_total": info.inner_total,
            "relres": info.relres,
            "seconds": time.perf_counter() - t,
            "sample_inner_iters": SAMPLE_INNER[name],
            "sample_seconds": ts,
            "host_cpu": _cpu_name(),
            "threads": os.environ.get("OPENBLAS_NUM_THREADS", "unset")}


def _cpu_name():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            data = json.load(fh)
    for name in names or list(SAMPLE_INNER):
        data[name] = run(name)
        print(name, data[name], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
