#!/usr/bin/env python3
"""Benchmark of the GB300 two-level-deflation Helmholtz solver.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--prec mixed_bf16|mixed|fp64]
                    [--basis16 0|1] [--autotune 0|1] [--cuda-graph 0|1]

A step is one complete solve of a batch of right-hand sides to relative
residual 1e-6 through the C ABI (hz_solve): outer FP64 flexible GMRES, the
A-DEF1 preconditioner with its inner coarse solve and V-cycles.  The metric
is unknowns * solves per second (whole job), device-timed with CUDA events;
``e2e`` repeats it through hz_solve_host with host buffers and the copies
inside the timed region.  Under torchrun every rank solves its own shots
(replicas, weak scaling; there is no exchange between ranks).

Default variant: complex-FP32 preconditioner with BF16-stored V-cycle
vectors and an FP16 inner Krylov basis, inside FP64 FGMRES (every solve
still reaches the FP64 true residual 1e-6, reported per step), with the
kernel choices of hz_autotune; ``fp64`` in the output line times the same
workload with the FP64 preconditioner.

``--impl reference`` times the CPU FP64 oracle (the plain restatement of the
method used by the tests) on a bounded sample of the same workload.
"""

import os

for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import tempfile  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unknowns*solves/s to rel.res 1e-6"
UNIT = "unknowns*solves/s"

# Workloads (seeded, synthetic).  mp2b: unit square, constant k, Sommerfeld
# boundaries, kh = 0.625; 16 point sources on a lattice around the centre.
WORKLOADS = {
    "mp2b_1281_k800_b16": dict(model=("constant_k", 1281, 800.0),
                               bc="sommerfeld", z="ho", e="galerkin",
                               nrhs=16, sources="centre_cluster",
                               coarse_tol=1e-1, coarse_maxit=200,
                               outer_maxit=60, tol=1e-6),
    "mp2b_641_k400_b16": dict(model=("constant_k", 641, 400.0),
                              bc="sommerfeld", z="ho", e="galerkin",
                              nrhs=16, sources="centre_cluster",
                              coarse_tol=1e-1, coarse_maxit=200,
                              outer_maxit=60, tol=1e-6),
    # small case for ncu captures (about 2.5 GB of workspace)
    "mp2b_641_k400_b8_prof": dict(model=("constant_k", 641, 400.0),
                                  bc="sommerfeld", z="ho", e="galerkin",
                                  nrhs=8, sources="centre_cluster",
                                  coarse_tol=1e-1, coarse_maxit=120,
                                  outer_maxit=16, tol=1e-6),
    "mp2a_81_k50": dict(model=("constant_k", 81, 50.0), bc="dirichlet",
                        z="bilinear", e="galerkin", nrhs=1,
                        sources="centre", coarse_tol=1e-6,
                        coarse_maxit=1000, outer_maxit=100, tol=1e-6),
    # three-layer wedge, 40 Hz on 289 x 481 (h = 2.08 m, kh = 0.35 at
    # 1500 m/s), one source on the surface at x = 300 m
    "wedge_289x481_f40": dict(model=("wedge", 289, 481, 40.0),
                              bc="sommerfeld", z="ho", e="galerkin", nrhs=1,
                              sources="surface_mid", coarse_tol=1e-1,
                              coarse_maxit=200, outer_maxit=60, tol=1e-6),
    # seeded layered-and-faulted model, 2301 x 751 physical nodes (h = 4 m)
    # padded to 2305 x 769, 31.25 Hz (kh = 0.52 at 1500 m/s), 64 surface
    # sources at i = 35 + 35 s
    "layered_2305x769_b64": dict(model=("layered", 2301, 751, 31.25),
                                 bc="sommerfeld", z="ho", e="galerkin",
                                 nrhs=64, sources="surface_line",
                                 coarse_tol=1e-1, coarse_maxit=160,
                                 outer_maxit=30, tol=1e-6),
    # the same model with 4 shots, for ncu captures (about 6 GB of workspace)
    "layered_2305x769_b4_prof": dict(model=("layered", 2301, 751, 31.25),
                                     bc="sommerfeld", z="ho", e="galerkin",
                                     nrhs=4, sources="surface_line",
                                     coarse_tol=1e-1, coarse_maxit=160,
                                     outer_maxit=4, tol=1e-6),
}
DEFAULT_WORKLOAD = "layered_2305x769_b64"
ORACLE_COUNTS = os.path.join(ROOT, "tests", "golden", "oracle_bench_counts.json")
ORACLE_COUNT_KEY = {"mp2b_1281_k800_b16": "mp2b_1281_k800",
                    "mp2a_81_k50": "mp2a_81_k50",
                    "layered_2305x769_b64": "layered_2305x769_b64"}


def rank_sources(nodes, rank):
    """Shots of one replica: the workload's source lattice shifted by the
    rank along x, so that every rank solves different right-hand sides."""
    return [(i + rank, j) for (i, j) in nodes] if rank else list(nodes)


def max_over_ranks(value, world, device="cpu"):
    """Max of a per-rank float over all ranks (the job's wall time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_inputs(wl_name, rank=0):
    from paper_2308_06152_gb300 import workloads as wl
    cfg = WORKLOADS[wl_name]
    kind = cfg["model"][0]
    if kind == "constant_k":
        model = wl.constant_k(*cfg["model"][1:])
    elif kind == "wedge":
        _, nx, ny, f = cfg["model"]
        model = wl.wedge(f, nx, ny)
    else:
        _, nx, ny, f = cfg["model"]
        model = wl.layered_faulted(nx, ny, freq=f)
    if cfg["sources"] == "centre":
        nodes = [wl.centre_node(model.nx, model.ny)] * cfg["nrhs"]
    elif cfg["sources"] == "surface_mid":
        nodes = rank_sources([((model.nx - 1) // 2, 0)] * cfg["nrhs"], rank)
    elif cfg["sources"] == "surface_line":
        nodes = rank_sources(wl.surface_line(model.physical[0] - 1,
                                             cfg["nrhs"]), rank)
    else:
        nodes = rank_sources(wl.centre_cluster(model.nx, model.ny,
                                               cfg["nrhs"]), rank)
    b = wl.point_sources(model.nx, model.ny, nodes)
    return cfg, model, b


def unknowns(cfg, model):
    """Unknowns per solve; a padded model counts its physical nodes only."""
    if cfg["bc"] == "dirichlet":
        return (model.nx - 2) * (model.ny - 2)
    return model.physical[0] * model.physical[1]


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid=None):
        self.proc = None
        self.path = None
        self.uuid = dev_uuid

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}",
               "--format=csv,noheader,nounits", "-lms", "200",
               "-f", self.path]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap")
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        load = [v for v in sm if mx and v > 0.5 * max(mx)] or sm
        return {"sm_mhz": float(np.median(load)) if load else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons}


PREC_TEXT = {"mixed": "complex-FP32 preconditioner in FP64 FGMRES",
             "mixed_bf16": ("complex-FP32 preconditioner with BF16-storage "
                            "V-cycle vectors, in FP64 FGMRES"),
             "fp64": "complex-FP64 throughout"}

KERNEL_NAMES = {"mdot": "k_mdot (CGS2 multi-vector dot product)",
                "maxpy": "k_maxpy (CGS2 multi-vector update)",
                "vcycle": ("k_pre_restrict_mr + k_prolong_smooth_mr / _cell (top "
                           "level of every V-cycle, staged form)")}


def hbm_peak():
    """Measured HBM copy bandwidth of the GB300s, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle
def _oracle_recorded(wl_name):
    key = ORACLE_COUNT_KEY.get(wl_name)
    if not key or not os.path.exists(ORACLE_COUNTS):
        return key, None
    with open(ORACLE_COUNTS) as fh:
        rec = json.load(fh).get(key)
    if rec and "sample_seconds" in rec and "seconds" in rec:
        return key, rec
    return key, None


def _oracle_sample_worker(key):
    """Set up the oracle for the workload's first shot and time its
    calibration sample once (one spawned process per host core)."""
    from oracle.record_bench_counts import (SAMPLE_INNER, calibration_sample,
                                            make_oracle)
    orc, b, _ = make_oracle(key)
    return calibration_sample(orc, b, SAMPLE_INNER[key])


def oracle_sample(wl_name, steps, warmup, all_cores=False):
    """CPU baseline: the FP64 oracle (SciPy CSR, one core) on the
    workload's first shot.  A whole oracle solve of that shot was timed by
    oracle/record_bench_counts.py, together with a bounded calibration
    sample (the first coarse solve, stopped after a fixed number of inner
    iterations) in the same process.  Here the same sample is timed again
    on this host (``warmup`` untimed and ``steps`` timed repetitions), and
    the recorded whole-solve time is carried over to this host by the ratio
    of the two sample times.  With all_cores the sample also runs in one
    spawned process per host core at once (each its own copy of the shot),
    and the batched figure uses the per-process sample time."""
    cfg, model, _ = build_inputs(wl_name)
    n_unk = unknowns(cfg, model)
    key, rec = _oracle_recorded(wl_name)
    if rec is None:
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"no recorded whole oracle solve for {wl_name}"}
    from oracle.record_bench_counts import (SAMPLE_INNER, calibration_sample,
                                            make_oracle)
    t0 = time.perf_counter()
    orc, b, _ = make_oracle(key)
    t_setup = time.perf_counter() - t0
    times = []
    for it in range(warmup + steps):
        dt = calibration_sample(orc, b, SAMPLE_INNER[key])
        if it >= warmup:
            times.append(dt)
    del orc
    t_s = float(np.mean(times))
    scale = t_s / rec["sample_seconds"]
    t_full = rec["seconds"] * scale
    out = {"value": n_unk / t_full, "unit": UNIT, "cores": 1, "kind": "oracle",
           "arithmetic": "FP64 throughout (SciPy CSR), the oracle's own "
                         "iteration counts",
           "seconds_per_solve": t_full,
           "sample": (f"one shot of {wl_name} (its first source). Timed whole "
                      f"oracle solve: {rec['seconds']:.1f} s, "
                      f"{rec['outer_iters']} outer / {rec['inner_iters_total']} "
                      f"inner iterations, on {rec.get('host_cpu', 'the recording host')} "
                      f"(oracle/record_bench_counts.py); carried to this host "
                      f"({_host_cpu()}) by a calibration sample (the first "
                      f"coarse solve stopped after {SAMPLE_INNER[key]} inner "
                      f"iterations): {t_s:.2f} s here against "
                      f"{rec['sample_seconds']:.2f} s there (mean of {len(times)} "
                      f"after {warmup} untimed; set-up {t_setup:.1f} s not "
                      f"counted), so {t_full:.0f} s per solve here")}
    if all_cores:
        import multiprocessing as mp
        procs = os.cpu_count() or 1
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_sample_worker, [key] * procs)
        wall = time.perf_counter() - t0
        t_par = float(np.mean(res))
        t_full_par = rec["seconds"] * t_par / rec["sample_seconds"]
        out["all_cores"] = {
            "value": n_unk * procs / t_full_par, "unit": UNIT, "cores": procs,
            "sample": (f"the calibration sample in {procs} spawned processes at "
                       f"once, one shot each: {t_par:.2f} s per process "
                       f"({wall:.0f} s wall incl. set-up), so "
                       f"{t_full_par:.0f} s per solve per core")}
    return out


def _host_cpu():
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def workload_config(args, cfg, model, world, b_np):
    """The "config" of the output line shared by both arms: what the
    workload is and how it is solved."""
    return {"workload": args.workload, "grid": [model.nx, model.ny],
            "physical_grid": list(model.physical),
            "velocity_model": model.name,
            "kh_max": round(model.kh_max(), 4), "bc": cfg["bc"],
            "deflation": f"{cfg['z']}/{cfg['e']}",
            "outer": args.outer, "preconditioner": args.precond,
            "precision": PREC_TEXT[args.prec],
            "inner_basis_storage": ("fp16" if args.basis16 and args.prec != "fp64"
                                    else ("c64" if args.prec != "fp64" else "c128")),
            "nrhs_per_gpu": cfg["nrhs"], "tol": cfg["tol"],
            "coarse_tol": cfg["coarse_tol"],
            "parallelism": f"replicas{world}",
            "l2": ("inputs larger than L2 (each batch vector "
                   f"{b_np.nbytes / 1e6:.0f} MB)")}


# DRAM bytes / algorithmic bytes of a profiled kernel class, measured with
# ncu on the same kernel and storage (the summary under profiles/ names the
# command); traffic scales with the rows streamed, so a bench launch's
# traffic is this ratio times its algorithmic bytes.
TRAFFIC = {
    ("mdot", "layered_2305x769_b64", 0): (1.004, "profiles/dram_layered_2305x769_b64.md"),
    ("maxpy", "layered_2305x769_b64", 0): (1.006, "profiles/dram_layered_2305x769_b64.md"),
    ("vcycle", "layered_2305x769_b64", (2, 8, 0)): (
        0.885, "profiles/dram_layered_2305x769_b64.md"),
    ("vcycle", "layered_2305x769_b64", (2, 16, 0)): (
        0.889, "profiles/dram_layered_2305x769_b64.md"),
}


def roofline_entry(args, tuning, kc, prof, prof_ms):
    if not prof or prof[0] <= 0:
        return None
    n_l, ms_k, by = prof
    peak, peak_src = hbm_peak()
    achieved = by / (ms_k / 1e3) / 1e9
    ratio = TRAFFIC.get((kc, args.workload, _variant(kc, tuning)))
    return {"kernel": KERNEL_NAMES[kc], "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": (ratio[0] * by / n_l if ratio else None),
            "traffic_source": (ratio[1] if ratio else None),
            "launches": int(n_l),
            "alg_bytes_per_launch": by / n_l,
            "avg_launch_us": 1e3 * ms_k / n_l,
            "timed_over": (f"{args.profile_steps} further step(s) of the "
                           "same workload with the kernels issued one by "
                           "one (events around each launch)"),
            "profiled_step_ms": prof_ms,
            "share_of_step": ms_k / (prof_ms * args.profile_steps)}


def _variant(kc, tuning):
    if kc == "mdot":
        return tuning.get("mdot_kernel")
    if kc == "maxpy":
        return tuning.get("maxpy_kernel")
    if kc == "vcycle":
        return (tuning.get("vcycle_fused"), tuning.get("vcycle_rhs_per_block"),
                tuning.get("vcycle_tile"))
    return None


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2308_06152_gb300._lib import load_library
    from paper_2308_06152_gb300.api import Desc, Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lib = load_library()
    cfg, model, b_np = build_inputs(args.workload, rank)
    cfg = dict(cfg)
    for key in ("coarse_tol", "coarse_maxit", "outer_maxit"):
        if getattr(args, key) is not None:
            cfg[key] = getattr(args, key)
    desc = Desc(model.nx, model.ny, model.h, bc=cfg["bc"], z=cfg["z"],
                e=cfg["e"], prec=args.prec, nrhs_max=cfg["nrhs"],
                coarse_tol=cfg["coarse_tol"], coarse_maxit=cfg["coarse_maxit"],
                outer_maxit=cfg["outer_maxit"],
                inner_basis_fp16=bool(args.basis16),
                outer=args.outer, precond=args.precond,
                cuda_graph=bool(args.cuda_graph))
    solver = Solver(desc, model.k2)
    tune_ms = None
    if args.autotune:
        tune_ms = solver.autotune(cfg["nrhs"])["ms"]
    if args.mdot_kernel is not None:
        solver.set_tuning(mdot_kernel=args.mdot_kernel)
    if args.maxpy_kernel is not None:
        solver.set_tuning(maxpy_kernel=args.maxpy_kernel)
    if args.galerkin_apply is not None:
        solver.set_tuning(galerkin_apply=args.galerkin_apply)
    if args.vcycle_fused is not None:
        solver.set_tuning(vcycle_fused=args.vcycle_fused)
    if args.vcycle_rpb is not None:
        solver.set_tuning(vcycle_rhs_per_block=args.vcycle_rpb)
    if args.vcycle_tile is not None:
        solver.set_tuning(vcycle_tile=args.vcycle_tile)
    if args.e_pairs is not None:
        solver.set_tuning(e_column_pairs=args.e_pairs)
    tuning = solver.get_tuning()
    stream = solver.stream
    b = torch.from_numpy(b_np).cuda()
    tol = cfg["tol"]
    for _ in range(args.warmup):
        x, info = solver.solve(b, tol=tol)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        uuid = None
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    l0 = lib.hz_kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        x, info = solver.solve(b, tol=tol)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = lib.hz_kernel_launches() - l0
    # per-kernel timing: CUDA events must bracket every launch of the
    # profiled kernel class, which a replayed graph does not allow, so these
    # steps issue the same kernels one by one
    profs = []
    classes = [c for c in args.profile_kernel.split(",") if c and c != "none"]
    for kc in classes:
        solver.profile_begin(kc, max_launches=200000)
        pe0 = torch.cuda.Event(enable_timing=True)
        pe1 = torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        for _ in range(args.profile_steps):
            solver.solve(b, tol=tol)
        pe1.record(stream)
        torch.cuda.synchronize()
        profs.append((kc, solver.profile_end(),
                      pe0.elapsed_time(pe1) / args.profile_steps))
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, "cuda")
    if world > 1:
        dist.barrier()
    n_unk = unknowns(cfg, model)
    units = n_unk * cfg["nrhs"] * world
    value = units / (ms / 1000.0)
    worst = max(i.relres for step in infos for i in step)
    statuses = sorted({i.status for step in infos for i in step})
    outer = [i.outer_iters for i in infos[-1]]
    inner = [i.inner_iters_total for i in infos[-1]]

    # end to end through the host-buffer entry point
    bh = torch.from_numpy(b_np).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    solver.solve_host(bh, xh, tol=tol)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve_host(bh, xh, tol=tol)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world,
                           "cuda")
    io_bytes = int(b_np.nbytes)

    roofs = [roofline_entry(args, tuning, kc, prof, prof_ms)
             for kc, prof, prof_ms in profs]
    roofs = [r for r in roofs if r]
    roof = roofs[0] if roofs else None

    fp64 = None
    if args.compare_fp64 and args.prec != "fp64":
        # the same workload's first shots with the preconditioner in FP64
        # (one untimed and one timed solve); a sub-batch bounds the run time
        # of this roughly 16x slower form
        solver.close()
        del solver
        torch.cuda.synchronize()
        import dataclasses
        nsub = max(1, min(cfg["nrhs"], args.fp64_shots))
        s64 = Solver(dataclasses.replace(desc, prec="fp64", inner_basis_fp16=False,
                                         nrhs_max=nsub), model.k2)
        b64 = b[:nsub].contiguous()
        s64.solve(b64, tol=tol)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s64.stream)
        _, info64 = s64.solve(b64, tol=tol)
        e1.record(s64.stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        units64 = n_unk * nsub * world
        fp64 = {"value": units64 / (ms64 / 1e3), "unit": UNIT,
                "ms_per_step": ms64, "steps": 1, "warmup": 1,
                "shots": nsub,
                "sub_batch": (f"the first {nsub} of the workload's "
                              f"{cfg['nrhs']} shots in one batch"),
                "outer_iters": [i.outer_iters for i in info64],
                "max_true_relres": max(i.relres for i in info64),
                "mixed_over_fp64": value / (units64 / (ms64 / 1e3))}
        s64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_sample(args.workload, steps=1, warmup=0, all_cores=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c128" if args.prec == "fp64" else "c64",
            "data": "synthetic",
            "config": dict(workload_config(args, cfg, model, world, b_np),
                           cuda_graph=bool(args.cuda_graph), tuning=tuning,
                           autotune_ms=tune_ms),
            "e2e": {"value": units / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roof,
            "roofline_more": roofs[1:],
            "cpu_baseline": cpu,
            "fp64": fp64,
            "solve": {"outer_iters": outer, "inner_iters_total": inner,
                      "max_true_relres": worst, "status": statuses},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_kernel_bench(args):
    """V-cycle kernels alone at the size they run at inside the workload's
    inner solve: a solver on the workload's deflation coarse grid (level 1:
    ((nx+1)/2) x ((ny+1)/2) nodes, spacing 2h, the injected k^2), without
    deflation and with one-vector Krylov bases, so one V-cycle from its
    level 0 is the inner solve's V-cycle (FP32 input and output, the
    workload's level storage) on about 2.5 GB of device memory.  Prints
    the autotuner's time per V-cycle for every V-cycle candidate, then
    applies --kb-reps V-cycles with the tuning given on the command line
    (for ncu captures of single kernels)."""
    import torch

    from paper_2308_06152_gb300.api import Desc, Solver
    torch.cuda.set_device(0)
    cfg, model, _ = build_inputs(args.workload)
    k2c = np.ascontiguousarray(model.k2[::2, ::2])
    ny1, nx1 = k2c.shape
    nrhs = cfg["nrhs"]
    s = Solver(Desc(nx1, ny1, 2 * model.h, bc=cfg["bc"], z=None, e="galerkin",
                    prec=args.prec, nrhs_max=nrhs, coarse_maxit=1, outer_maxit=1,
                    inner_basis_fp16=bool(args.basis16)), k2c)
    vc = None
    if args.autotune:
        ms = s.autotune(nrhs)["ms"]
        vc = {k: v for k, v in ms.items() if k.startswith("vcycle")}
    choice = {}
    for key, val in (("vcycle_fused", args.vcycle_fused),
                     ("vcycle_rhs_per_block", args.vcycle_rpb),
                     ("vcycle_tile", args.vcycle_tile)):
        if val is not None:
            choice[key] = val
    if choice:
        s.set_tuning(**choice)
    f = torch.zeros((nrhs, ny1, nx1), dtype=torch.complex128, device="cuda")
    f[:, ny1 // 2, nx1 // 2] = 1.0
    for _ in range(args.kb_reps):
        s.apply("vcycle", f, 0)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_bench": "vcycle", "workload": args.workload,
                      "grid": [nx1, ny1], "nrhs": nrhs, "levels": s.num_levels,
                      "vcycle_ms": vc, "tuning": s.get_tuning()}), flush=True)
    s.close()


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cpu = oracle_sample(args.workload, steps=args.steps, warmup=args.warmup)
    cfg, model, b_np = build_inputs(args.workload)
    line = {
        "impl": "reference", "metric": METRIC, "value": cpu["value"],
        "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": workload_config(args, cfg, model, world, b_np),
        "cpu_baseline": cpu,
        "e2e": {"value": cpu["value"], "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS))
    ap.add_argument("--prec", choices=["mixed", "mixed_bf16", "fp64"],
                    default="mixed_bf16")
    ap.add_argument("--basis16", type=int, default=1,
                    help="store the inner coarse-solve Krylov basis as FP16")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU oracle baseline sample")
    ap.add_argument("--compare-fp64", type=int, default=1,
                    help="also time one solve with the FP64 preconditioner")
    ap.add_argument("--cuda-graph", type=int, default=1,
                    help="1: outer iterations as CUDA graphs with a device-side "
                         "inner WHILE loop; 0: kernels issued one by one")
    ap.add_argument("--outer", choices=["fgmres", "gcr"], default="fgmres",
                    help="outer Krylov iteration (hz_desc.outer_solver)")
    ap.add_argument("--precond", choices=["adef1", "tlkm"], default="adef1",
                    help="two-level preconditioner (hz_desc.preconditioner)")
    ap.add_argument("--coarse-tol", type=float, default=None,
                    help="override the workload's inner coarse-solve tolerance")
    ap.add_argument("--coarse-maxit", type=int, default=None,
                    help="override the inner iteration cap")
    ap.add_argument("--outer-maxit", type=int, default=None,
                    help="override the outer iteration cap")
    ap.add_argument("--autotune", type=int, default=1,
                    help="time the hz_tuning candidates at setup and keep the "
                         "fastest (outside the timed region)")
    ap.add_argument("--mdot-kernel", type=int, choices=[0, 1, 2], default=None,
                    help="force hz_tuning.mdot_kernel")
    ap.add_argument("--maxpy-kernel", type=int, choices=[0, 1, 2], default=None,
                    help="force hz_tuning.maxpy_kernel")
    ap.add_argument("--galerkin-apply", type=int, choices=[0, 1], default=None,
                    help="force hz_tuning.galerkin_apply")
    ap.add_argument("--vcycle-fused", type=int, choices=[0, 1, 2], default=None,
                    help="force hz_tuning.vcycle_fused")
    ap.add_argument("--vcycle-rpb", type=int, default=None,
                    help="force hz_tuning.vcycle_rhs_per_block")
    ap.add_argument("--vcycle-tile", type=int, choices=[0, 1], default=None,
                    help="force hz_tuning.vcycle_tile")
    ap.add_argument("--e-pairs", type=int, choices=[0, 1], default=None,
                    help="force hz_tuning.e_column_pairs")
    ap.add_argument("--profile-steps", type=int, default=1,
                    help="steps timed per kernel for the roofline entry")
    ap.add_argument("--profile-kernel", default="mdot,maxpy,vcycle",
                    help="comma-separated kernel classes (mdot, maxpy, vcycle) timed "
                         "live for the roofline entries (the first one is "
                         "'roofline', the others 'roofline_more'); 'none' "
                         "skips them")
    ap.add_argument("--fp64-shots", type=int, default=16,
                    help="shots of the FP64 comparison batch")
    ap.add_argument("--kernel-bench", action="store_true",
                    help="time the V-cycle kernels alone on the workload's "
                         "level-1 grid (see run_kernel_bench)")
    ap.add_argument("--kb-reps", type=int, default=3,
                    help="V-cycles applied by --kernel-bench after timing")
    args = ap.parse_args()
    if args.kernel_bench:
        run_kernel_bench(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
