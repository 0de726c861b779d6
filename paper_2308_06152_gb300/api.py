"""Python face of the C ABI: ``Desc`` (hz_desc) and ``Solver`` (hz_solver).

PyTorch provides device memory (the workspace, inputs, outputs) and the
CUDA stream; every operation is a call into libhz.so.
"""

import ctypes
from dataclasses import dataclass, field

import numpy as np
import torch

from ._lib import HzDesc, HzSolveInfo, HzTuning, STATUS, load_library

BC = {"dirichlet": 0, "sommerfeld": 1}
ZKIND = {None: 0, "none": 0, "bilinear": 1, "ho": 2}
EKIND = {"galerkin": 0, "red_o2": 1, "red_glk1": 2, "red_glk2": 3,
         "red_o4": 4, "red_cmpo4": 5, "red_o6": 6, "red_9pt": 7}
PREC = {"fp64": 0, "mixed": 1, "mixed_bf16": 2}
OUTER = {"fgmres": 0, "gcr": 1}
PRECOND = {"adef1": 0, "tlkm": 1}
DEFL_SCALE = {"consistent": 0, "printed": 1}
OPS = {"helmholtz": 0, "cslp": 1, "vcycle": 2, "restrict_fw": 3,
       "prolong_bilinear": 4, "restrict_z": 5, "prolong_z": 6, "coarse_e": 7,
       "coarse_solve": 8, "precond": 9}
# (input level offset, output level offset) relative to `level`
_OP_LEVELS = {"helmholtz": (0, 0), "cslp": (0, 0), "vcycle": (0, 0),
              "restrict_fw": (0, 1), "prolong_bilinear": (1, 0),
              "restrict_z": (0, 1), "prolong_z": (1, 0), "coarse_e": (1, 1),
              "coarse_solve": (1, 1), "precond": (0, 0)}


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


@dataclass
class Desc:
    nx: int
    ny: int
    h: float
    bc: str = "sommerfeld"
    z: object = "ho"
    e: str = "galerkin"
    prec: str = "fp64"
    beta: tuple = (1.0, -0.5)
    jacobi_omega: float = 0.8
    min_coarse_intervals: int = 2
    coarse_tol: float = 1e-6
    coarse_maxit: int = 500
    outer_maxit: int = 100
    nrhs_max: int = 1
    inner_basis_fp16: bool = False
    outer: str = "fgmres"
    precond: str = "adef1"
    deflation_levels: int = 1
    cuda_graph: bool = True
    deflation_scaling: str = "consistent"
    restart: int = 0

    def to_c(self):
        d = HzDesc()
        d.nx, d.ny, d.h = int(self.nx), int(self.ny), float(self.h)
        d.bc = BC[self.bc]
        d.zkind = ZKIND[self.z]
        d.ekind = EKIND[self.e]
        d.prec = PREC[self.prec]
        d.beta1, d.beta2 = float(self.beta[0]), float(self.beta[1])
        d.jacobi_omega = float(self.jacobi_omega)
        d.min_coarse_intervals = int(self.min_coarse_intervals)
        d.coarse_tol = float(self.coarse_tol)
        d.coarse_maxit = int(self.coarse_maxit)
        d.outer_maxit = int(self.outer_maxit)
        d.nrhs_max = int(self.nrhs_max)
        d.inner_basis_fp16 = int(bool(self.inner_basis_fp16))
        d.outer_solver = OUTER[self.outer]
        d.preconditioner = PRECOND[self.precond]
        d.deflation_levels = int(self.deflation_levels)
        d.no_cuda_graph = int(not self.cuda_graph)
        d.deflation_scaling = DEFL_SCALE[self.deflation_scaling]
        d.restart = int(self.restart)
        return d


def workspace_bytes(desc):
    lib = load_library()
    n = ctypes.c_size_t(0)
    cd = desc.to_c()
    st = lib.hz_workspace_bytes(ctypes.byref(cd), ctypes.byref(n))
    if st != 0:
        raise HzError(st, "hz_workspace_bytes rejected the descriptor")
    return n.value


@dataclass
class Info:
    outer_iters: int
    inner_iters_total: int
    inner_iters_max: int
    relres: float
    status: str
    extra: dict = field(default_factory=dict)


def _infos(arr, n):
    return [Info(arr[i].outer_iters, arr[i].inner_iters_total,
                 arr[i].inner_iters_max, arr[i].relres,
                 STATUS.get(arr[i].status, str(arr[i].status)))
            for i in range(n)]


class Solver:
    """A set-up solver bound to one grid, wavenumber field and stream.

    ``k2``: (ny, nx) squared wavenumber (numpy or torch; copied to the
    device).  The workspace is a torch uint8 tensor owned by the solver.
    """

    def __init__(self, desc, k2, device=None, stream=None, workspace=None):
        self.lib = load_library()
        self.desc = desc
        dev = torch.device(device) if device is not None else \
            torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.stream = stream if stream is not None else \
            torch.cuda.current_stream(dev)
        k2t = torch.as_tensor(np.asarray(k2) if not torch.is_tensor(k2) else k2,
                              dtype=torch.float64).reshape(desc.ny, desc.nx)
        self.k2 = k2t.to(dev).contiguous()
        self.ws_bytes = workspace_bytes(desc)
        if workspace is None:
            workspace = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.ws = workspace
        cd = desc.to_c()
        handle = ctypes.c_void_p()
        st = self.lib.hz_setup(ctypes.byref(cd), self.k2.data_ptr(),
                               self.ws.data_ptr(),
                               ctypes.c_size_t(self.ws.numel()),
                               self.stream.cuda_stream, ctypes.byref(handle))
        if st != 0:
            raise HzError(st, "hz_setup failed")
        self.handle = handle

    # ------------------------------------------------------------ helpers
    def _check(self, st, what):
        if st not in (0,):
            msg = self.lib.hz_last_error(self.handle)
            raise HzError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def num_levels(self):
        return self.lib.hz_num_levels(self.handle)

    def level_shape(self, level):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.hz_level_shape(self.handle, level, ctypes.byref(nx),
                                            ctypes.byref(ny)), "level_shape")
        return nx.value, ny.value

    def _rhs(self, b):
        b = torch.as_tensor(b)
        if b.dim() == 2:
            b = b.unsqueeze(0)
        return b.to(device=self.device, dtype=torch.complex128).contiguous()

    # ------------------------------------------------------------ solve
    def solve(self, b, tol=1e-6, x0=None, raise_on_fail=False):
        """x, infos = solve(b): b complex (nrhs, ny, nx) on the device."""
        b = self._rhs(b)
        nrhs = b.shape[0]
        if x0 is None:
            x = torch.empty_like(b)
            use_x0 = 0
        else:
            x = self._rhs(x0).clone()
            use_x0 = 1
        infos = (HzSolveInfo * nrhs)()
        st = self.lib.hz_solve(self.handle, b.data_ptr(), x.data_ptr(), nrhs,
                               float(tol), use_x0, infos)
        if st not in (0, 4, 5, 6) or (raise_on_fail and st != 0):
            self._check(st, "hz_solve")
        return x, _infos(infos, nrhs)

    def solve_async(self, b, tol=1e-6, x0=None):
        """x, info_dev = solve_async(b): enqueues the whole solve as one CUDA
        graph (hz_solve_async) and returns at once; info_dev is a device
        buffer of nrhs hz_solve_info records (read it with infos_from_device
        after the stream reached the end of the solve)."""
        b = self._rhs(b)
        nrhs = b.shape[0]
        if x0 is None:
            x = torch.empty_like(b)
            use_x0 = 0
        else:
            x = self._rhs(x0).clone()
            use_x0 = 1
        info = torch.zeros(nrhs * ctypes.sizeof(HzSolveInfo), dtype=torch.uint8,
                           device=self.device)
        self._check(self.lib.hz_solve_async(self.handle, b.data_ptr(), x.data_ptr(), nrhs,
                                            float(tol), use_x0, info.data_ptr()),
                    "hz_solve_async")
        return x, info

    @staticmethod
    def infos_from_device(info):
        """The hz_solve_info records of a device buffer (copies to the host)."""
        raw = info.cpu().numpy().tobytes()
        nrhs = len(raw) // ctypes.sizeof(HzSolveInfo)
        recs = (HzSolveInfo * nrhs).from_buffer_copy(raw)
        return _infos(recs, nrhs)

    def solve_host(self, b_host, x_host=None, tol=1e-6):
        """End-to-end solve from and to host (ideally pinned) memory."""
        nrhs = b_host.shape[0]
        if x_host is None:
            x_host = torch.empty_like(b_host)
        infos = (HzSolveInfo * nrhs)()
        st = self.lib.hz_solve_host(self.handle, b_host.data_ptr(),
                                    x_host.data_ptr(), nrhs, float(tol), infos)
        if st not in (0, 4, 5, 6):
            self._check(st, "hz_solve_host")
        return x_host, _infos(infos, nrhs)

    def apply(self, op, x, level=0):
        """y = op(x) for one operator of the method (see hz_op)."""
        x = self._rhs(x)
        nrhs = x.shape[0]
        _, lo = _OP_LEVELS[op]
        nxo, nyo = self.level_shape(level + lo)
        y = torch.empty((nrhs, nyo, nxo), dtype=torch.complex128,
                        device=self.device)
        self._check(self.lib.hz_apply(self.handle, OPS[op], level, x.data_ptr(),
                                      y.data_ptr(), nrhs), f"hz_apply({op})")
        return y

    def last_inner_iters(self, nrhs):
        out = (ctypes.c_int * nrhs)()
        self._check(self.lib.hz_last_inner_iters(self.handle, out, nrhs),
                    "last_inner_iters")
        return list(out)

    def gradient(self, omega, src, rec_idx, d_obs, tol=1e-10):
        """J, grad (ny, nx) float64 device tensor, infos (2 per shot)."""
        src = self._rhs(src)
        nshots = src.shape[0]
        rec = torch.as_tensor(rec_idx, dtype=torch.int32).to(self.device)
        d = torch.as_tensor(d_obs).to(device=self.device,
                                      dtype=torch.complex128).contiguous()
        grad = torch.empty((self.desc.ny, self.desc.nx), dtype=torch.float64,
                           device=self.device)
        J = ctypes.c_double(0.0)
        infos = (HzSolveInfo * (2 * nshots))()
        st = self.lib.hz_gradient(self.handle, float(omega), src.data_ptr(),
                                  nshots, rec.data_ptr(), rec.numel(),
                                  d.data_ptr(), float(tol), ctypes.byref(J),
                                  grad.data_ptr(), infos)
        if st not in (0, 4, 5):
            self._check(st, "hz_gradient")
        return J.value, grad, _infos(infos, 2 * nshots)

    KERNEL_CLASSES = {"mdot": 1, "maxpy": 2, "vcycle": 3}

    def profile_begin(self, kernel, max_launches=100000):
        """Time every launch of one kernel class (see hz_profile_begin)."""
        self._check(self.lib.hz_profile_begin(self.handle,
                                              self.KERNEL_CLASSES[kernel],
                                              int(max_launches)),
                    "hz_profile_begin")

    def profile_end(self):
        """(launches, total ms, algorithmic bytes) since profile_begin."""
        n = ctypes.c_longlong(0)
        ms = ctypes.c_double(0.0)
        by = ctypes.c_double(0.0)
        self._check(self.lib.hz_profile_end(self.handle, ctypes.byref(n),
                                            ctypes.byref(ms),
                                            ctypes.byref(by)),
                    "hz_profile_end")
        return n.value, ms.value, by.value

    def get_tuning(self):
        """The solver's implementation choices as a dict (see hz_tuning)."""
        t = HzTuning()
        self._check(self.lib.hz_get_tuning(self.handle, ctypes.byref(t)),
                    "hz_get_tuning")
        return {f: getattr(t, f) for f, _ in HzTuning._fields_}

    def set_tuning(self, **choices):
        """Set some or all hz_tuning fields; the others keep their values."""
        t = HzTuning()
        self._check(self.lib.hz_get_tuning(self.handle, ctypes.byref(t)),
                    "hz_get_tuning")
        for k, v in choices.items():
            if k not in dict(HzTuning._fields_):
                raise KeyError(f"unknown tuning field {k}")
            setattr(t, k, int(v))
        self._check(self.lib.hz_set_tuning(self.handle, ctypes.byref(t)),
                    "hz_set_tuning")

    TUNE_CANDIDATES = ("mdot_kernel=0", "mdot_kernel=1", "mdot_kernel=2",
                       "maxpy_kernel=0", "maxpy_kernel=1", "maxpy_kernel=2",
                       "galerkin_apply=0", "galerkin_apply=1",
                       "e_rhs_per_block=0", "e_rhs_per_block=8",
                       "e_rhs_per_block=4", "vcycle_fused=0",
                       "vcycle_fused=1",
                       "vcycle_fused=2,rpb=4,tile=0", "vcycle_fused=2,rpb=8,tile=0",
                       "vcycle_fused=2,rpb=16,tile=0", "vcycle_fused=2,rpb=4,tile=1",
                       "vcycle_fused=2,rpb=8,tile=1", "vcycle_fused=2,rpb=16,tile=1",
                       "e_column_pairs=1")

    def tuning_key(self, nrhs):
        """Cache key of a tuning: the device and every descriptor field
        that changes the timed kernels' shapes."""
        d = self.desc
        name = torch.cuda.get_device_name(self.device)
        return (f"{name}|{d.nx}x{d.ny}|bc={d.bc}|z={d.z}|e={d.e}|prec={d.prec}"
                f"|basis16={int(bool(d.inner_basis_fp16))}|nrhs={nrhs}"
                f"|maxit={d.coarse_maxit},{d.outer_maxit}")

    def autotune(self, nrhs=None, cache=None):
        """Pick the hz_tuning fields by timing them (hz_autotune) for nrhs
        right-hand sides (default nrhs_max).  With ``cache`` (a JSON file
        path) an earlier choice for the same key is reused without timing,
        and a new one is stored.  Returns {"tuning", "ms", "cached"}."""
        import json
        import os
        nrhs = int(nrhs or self.desc.nrhs_max)
        key = self.tuning_key(nrhs)
        data = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                data = json.load(fh)
            if key in data:
                self.set_tuning(**data[key]["tuning"])
                return dict(data[key], cached=True)
        t = HzTuning()
        ms = (ctypes.c_double * len(self.TUNE_CANDIDATES))()
        self._check(self.lib.hz_autotune(self.handle, nrhs, ctypes.byref(t), ms),
                    "hz_autotune")
        entry = {"tuning": {f: getattr(t, f) for f, _ in HzTuning._fields_},
                 "ms": {c: (ms[i] if ms[i] >= 0 else None)
                        for i, c in enumerate(self.TUNE_CANDIDATES)}}
        if cache:
            data[key] = entry
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(entry, cached=False)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hz_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptrs(values):
    arr = (ctypes.c_void_p * len(values))()
    for i, v in enumerate(values):
        arr[i] = v
    return arr


def solve_group(solvers, bs, tol=1e-6):
    """Solve on several solvers (grids of different sizes) together
    (hz_solve_group).  bs[g]: complex (nrhs_g, ny_g, nx_g).  Returns a list
    of (x_g, infos_g)."""
    lib = load_library()
    K = len(solvers)
    bs = [s._rhs(b) for s, b in zip(solvers, bs)]
    xs = [torch.empty_like(b) for b in bs]
    nrhs = (ctypes.c_int * K)(*[b.shape[0] for b in bs])
    infos = [(HzSolveInfo * b.shape[0])() for b in bs]
    st = lib.hz_solve_group(_ptrs([s.handle.value for s in solvers]), K,
                            _ptrs([b.data_ptr() for b in bs]),
                            _ptrs([x.data_ptr() for x in xs]), nrhs, float(tol),
                            _ptrs([ctypes.addressof(i) for i in infos]))
    if st not in (0, 4, 5, 6):
        solvers[0]._check(st, "hz_solve_group")
    return [(x, _infos(i, b.shape[0])) for x, i, b in zip(xs, infos, bs)]


def gradient_group(solvers, omegas, srcs, recs, ds, tol=1e-10):
    """hz_gradient over several grids at once: lists per member of omega,
    sources (nshots, ny, nx), receiver indices and data (nshots, nrec).
    Returns a list of (J_g, grad_g, infos_g)."""
    lib = load_library()
    K = len(solvers)
    srcs = [s._rhs(x) for s, x in zip(solvers, srcs)]
    recs = [torch.as_tensor(r, dtype=torch.int32).to(s.device)
            for s, r in zip(solvers, recs)]
    ds = [torch.as_tensor(d).to(device=s.device, dtype=torch.complex128).contiguous()
          for s, d in zip(solvers, ds)]
    grads = [torch.empty((s.desc.ny, s.desc.nx), dtype=torch.float64,
                         device=s.device) for s in solvers]
    J = (ctypes.c_double * K)()
    infos = [(HzSolveInfo * (2 * x.shape[0]))() for x in srcs]
    st = lib.hz_gradient_group(
        _ptrs([s.handle.value for s in solvers]), K,
        (ctypes.c_double * K)(*[float(o) for o in omegas]),
        _ptrs([x.data_ptr() for x in srcs]),
        (ctypes.c_int * K)(*[x.shape[0] for x in srcs]),
        _ptrs([r.data_ptr() for r in recs]),
        (ctypes.c_int * K)(*[r.numel() for r in recs]),
        _ptrs([d.data_ptr() for d in ds]), float(tol), J,
        _ptrs([g.data_ptr() for g in grads]),
        _ptrs([ctypes.addressof(i) for i in infos]))
    if st not in (0, 4, 5):
        solvers[0]._check(st, "hz_gradient_group")
    return [(J[g], grads[g], _infos(infos[g], 2 * srcs[g].shape[0]))
            for g in range(K)]
