"""ctypes loader of libhz.so and the C structs of include/hz.h.

Argument marshalling only; every step of the method runs in the library's
CUDA kernels.  There is no fallback: if libhz.so is missing the loader
raises.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhz.so")

c_int, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_size_t)


class HzDesc(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("h", c_double),
                ("bc", c_int), ("zkind", c_int), ("ekind", c_int),
                ("prec", c_int), ("beta1", c_double), ("beta2", c_double),
                ("jacobi_omega", c_double), ("min_coarse_intervals", c_int),
                ("coarse_tol", c_double), ("coarse_maxit", c_int),
                ("outer_maxit", c_int), ("nrhs_max", c_int),
                ("inner_basis_fp16", c_int),
                ("outer_solver", c_int),
                ("preconditioner", c_int),
                ("deflation_levels", c_int),
                ("no_cuda_graph", c_int),
                ("deflation_scaling", c_int), ("restart", c_int)]


class HzSolveInfo(ctypes.Structure):
    _fields_ = [("outer_iters", c_int), ("inner_iters_total", c_int),
                ("inner_iters_max", c_int), ("relres", c_double),
                ("status", c_int)]


class HzTuning(ctypes.Structure):
    _fields_ = [("mdot_kernel", c_int), ("maxpy_kernel", c_int),
                ("galerkin_apply", c_int), ("e_rhs_per_block", c_int),
                ("vcycle_fused", c_int), ("vcycle_rhs_per_block", c_int),
                ("vcycle_tile", c_int), ("e_column_pairs", c_int)]


STATUS = {0: "HZ_OK", 1: "HZ_INVALID_ARG", 2: "HZ_INVALID_GRID",
          3: "HZ_WORKSPACE_TOO_SMALL", 4: "HZ_NOT_CONVERGED",
          5: "HZ_BREAKDOWN", 6: "HZ_NAN", 7: "HZ_TIMEOUT",
          8: "HZ_CUDA_ERROR"}

# name -> (restype, argtypes)
SIGNATURES = {
    "hz_desc_default": (None, [c_void_p, c_int, c_int, c_double]),
    "hz_workspace_bytes": (c_int, [c_void_p, c_void_p]),
    "hz_setup": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t, c_void_p,
                         c_void_p]),
    "hz_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int,
                         c_void_p]),
    "hz_solve_async": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int,
                               c_void_p]),
    "hz_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_double,
                              c_void_p]),
    "hz_apply": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_int]),
    "hz_last_inner_iters": (c_int, [c_void_p, c_void_p, c_int]),
    "hz_num_levels": (c_int, [c_void_p]),
    "hz_level_shape": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "hz_gradient": (c_int, [c_void_p, c_double, c_void_p, c_int, c_void_p,
                            c_int, c_void_p, c_double, c_void_p, c_void_p,
                            c_void_p]),
    "hz_coarse_galerkin_noalloc": (c_int, [c_int, c_int, c_double, c_int,
                                           c_int, c_void_p, c_void_p,
                                           c_void_p, c_int, c_void_p]),
    "hz_destroy": (c_int, [c_void_p]),
    "hz_kernel_launches": (ctypes.c_longlong, []),
    "hz_host_launches": (ctypes.c_longlong, []),
    "hz_fault_drill": (c_int, [c_void_p, c_int, c_double]),
    "hz_profile_begin": (c_int, [c_void_p, c_int, c_int]),
    "hz_profile_end": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "hz_tuning_default": (None, [c_void_p]),
    "hz_get_tuning": (c_int, [c_void_p, c_void_p]),
    "hz_set_tuning": (c_int, [c_void_p, c_void_p]),
    "hz_autotune": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    "hz_solve_group": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p,
                               c_double, c_void_p]),
    "hz_gradient_group": (c_int, [c_void_p, c_int, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_double, c_void_p, c_void_p, c_void_p]),
    "hz_status_str": (ctypes.c_char_p, [c_int]),
    "hz_last_error": (ctypes.c_char_p, [c_void_p]),
}

_LIB = None


def load_library(path=None):
    """Load libhz.so (cached).  Raises RuntimeError if it was not built."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"{p} is missing: build it with "
            "`python -m paper_2308_06152_gb300.build` (needs nvcc); there is "
            "no CPU fallback")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _LIB = lib
    return lib
