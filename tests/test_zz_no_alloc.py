"""hz_coarse_galerkin_noalloc against the regular workspace path.

Some callers cannot allocate device memory: services whose device-memory
budget is fixed at start-up, plug-ins inside a host framework that owns all
device memory, loops that must not block in an allocator.  For them the
library offers the Galerkin coarse operator with its two fine-grid
intermediates in a fixed, library-owned device array.  Its result must be
the one hz_apply(HZ_OP_COARSE_E) gives on an FP64 solver set up with the
Galerkin coarse operator, within the FP64 operator tolerance of the other
tests (1e-12 relative), on consecutive calls.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest

from paper_2308_06152_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BC = {"dirichlet": 0, "sommerfeld": 1}
ZK = {"bilinear": 1, "ho": 2}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2308_06152_gb300 import _lib, build
    build.build()
    return _lib.load_library()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("bc,z", [("sommerfeld", "ho"),
                                  ("dirichlet", "bilinear")])
def test_noalloc_matches_workspace_path_on_two_calls(lib, bc, z):
    from paper_2308_06152_gb300.api import Desc, Solver
    nx, ny, h = 97, 73, 1.0 / 96
    k2 = np.random.default_rng(3).uniform(4.0, 30.0, size=(ny, nx)) ** 2
    s = Solver(Desc(nx, ny, h, bc=bc, z=z, e="galerkin", prec="fp64",
                    nrhs_max=2), k2)
    ncx, ncy = s.level_shape(1)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        x = torch.from_numpy(wl.random_complex((2, ncy, ncx), 40 + call)).cuda()
        ref = s.apply("coarse_e", x).cpu().numpy()
        y = torch.full_like(x, float("nan"))
        st = lib.hz_coarse_galerkin_noalloc(nx, ny, h, BC[bc], ZK[z],
                                            s.k2.data_ptr(), x.data_ptr(),
                                            y.data_ptr(), 2, stream)
        assert st == 0
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        for r in range(2):
            assert _rel(got[r], ref[r]) < 1e-12, (call, r)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    cap = 32 * 1024 * 1024
    nx = ny = 1025
    assert 2 * nx * ny * 16 > cap
    k2 = torch.ones((ny, nx), dtype=torch.float64, device="cuda")
    x = torch.zeros((1, 513, 513), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    st = lib.hz_coarse_galerkin_noalloc(nx, ny, 1.0 / 1024, 1, 2,
                                        k2.data_ptr(), x.data_ptr(),
                                        y.data_ptr(), 1, None)
    assert st == 3   # HZ_WORKSPACE_TOO_SMALL
    st = lib.hz_coarse_galerkin_noalloc(4, 5, 0.1, 1, 2, k2.data_ptr(),
                                        x.data_ptr(), y.data_ptr(), 1, None)
    assert st == 1   # HZ_INVALID_ARG (even node count)
