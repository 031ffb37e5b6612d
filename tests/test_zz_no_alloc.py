"""The allocation-free body-force entry point (for callers that cannot call
cudaMalloc: its device staging buffer is a fixed array inside the library)
gives the same per-body force and torque sums as ibm_body_forces, on two
calls in a row (the second call reuses the shared array and must not see the
first call's contents).  Collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import gpu_cases as gc
from gpu_cases import dev

pytestmark = pytest.mark.gpu


def _noalloc(lib, F, X, bid, n, centers, h, stream):
    centers = np.ascontiguousarray(centers, dtype=np.float64)
    out = np.zeros((centers.shape[0], 6))
    st = lib.ibm_body_forces_noalloc(
        F.data_ptr(), X.data_ptr(), bid.data_ptr(), n, centers.shape[0],
        centers.ctypes.data_as(C.POINTER(C.c_double)), h, C.c_void_p(stream.cuda_stream),
        out.ctypes.data_as(C.POINTER(C.c_double)))
    return st, out


def test_noalloc_matches_body_forces_twice(cuda_device):
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300.api import IBMSolver
    case = gc.ragged_multi()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    s.set_markers(dev(case.X))
    X = dev(case.X.ravel())
    bid = dev(case.body_id.astype(np.int32))
    rng = np.random.default_rng(42)
    for call in range(2):
        # different forces each call: a stale staging buffer would show up
        F = dev(rng.standard_normal(3 * case.N) * (10.0 ** call))
        ref = s.body_forces(F, X, bid, case.centers)
        st, out = _noalloc(s.lib, F, X, bid, case.N, case.centers, case.h, s.stream)
        assert st == _lib.IBM_OK
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-300)
    s.close()
    torch.cuda.synchronize()


def test_noalloc_rejects_too_many_bodies(cuda_device):
    import torch
    from paper_2501_15314_gb300 import _lib
    lib = _lib.load()
    F = torch.zeros(3, dtype=torch.float64, device="cuda")
    bid = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = 1025                                  # IBM_NOALLOC_MAX_BODIES + 1
    centers = np.zeros((nb, 3))
    out = np.zeros((nb, 6))
    st = lib.ibm_body_forces_noalloc(F.data_ptr(), F.data_ptr(), bid.data_ptr(), 1, nb,
                                     centers.ctypes.data_as(C.POINTER(C.c_double)), 0.1, None,
                                     out.ctypes.data_as(C.POINTER(C.c_double)))
    assert st == _lib.IBM_ERR_ARG


def test_noalloc_refuses_misaligned_and_host_pointers(cuda_device):
    # refused with IBM_ERR_ARG before any launch: a device pointer off its
    # 8-byte alignment, and host memory the kernel must not be given
    import torch
    from paper_2501_15314_gb300 import _lib
    lib = _lib.load()
    n = 8
    F = torch.zeros(3 * n + 1, dtype=torch.float64, device="cuda")
    X = torch.zeros(3 * n, dtype=torch.float64, device="cuda")
    bid = torch.zeros(n, dtype=torch.int32, device="cuda")
    Fh = torch.zeros(3 * n, dtype=torch.float64)
    centers = np.zeros((1, 3))
    out = np.zeros((1, 6))
    cp = centers.ctypes.data_as(C.POINTER(C.c_double))
    op = out.ctypes.data_as(C.POINTER(C.c_double))
    l0 = lib.ibm_kernel_launches()
    for f, x, b in ((F.data_ptr() + 4, X.data_ptr(), bid.data_ptr()),
                    (F.data_ptr(), X.data_ptr(), bid.data_ptr() + 2),
                    (Fh.data_ptr(), X.data_ptr(), bid.data_ptr())):
        assert lib.ibm_body_forces_noalloc(f, x, b, n, 1, cp, 0.1, None, op) == _lib.IBM_ERR_ARG
    assert lib.ibm_kernel_launches() == l0
    torch.cuda.synchronize()


def test_noalloc_at_the_body_limit(cuda_device):
    # IBM_NOALLOC_MAX_BODIES bodies, markers assigned at random, against the
    # context call on the same inputs, twice in a row
    import torch
    from paper_2501_15314_gb300 import _lib
    from paper_2501_15314_gb300.api import IBMSolver
    rng = np.random.default_rng(7)
    nb, nm = 1024, 5000
    case = gc.ragged_multi()
    s = IBMSolver(case.nx, case.ny, case.nz, case.h, Re=case.Re, dt=case.dt)
    Xh = case.X[:, rng.integers(0, case.N, nm)] + 1e-3 * rng.standard_normal((3, nm))
    s.set_markers(dev(np.ascontiguousarray(Xh)))
    X = dev(np.ascontiguousarray(Xh).ravel())
    bid = dev(rng.integers(0, nb, nm).astype(np.int32))
    centers = rng.uniform(0.3, 0.7, (nb, 3))
    for call in range(2):
        F = dev(rng.standard_normal(3 * nm) * (3.0 ** call))
        ref = s.body_forces(F, X, bid, centers)
        st, out = _noalloc(s.lib, F, X, bid, nm, centers, case.h, s.stream)
        assert st == _lib.IBM_OK
        np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-300)
    s.close()
    torch.cuda.synchronize()
