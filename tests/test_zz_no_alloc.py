"""The allocation-free line-smoothing entry point against the allocating one.

ellsolve_level_smooth_noalloc exists for callers that cannot call cudaMalloc:
code running inside a CUDA stream capture, callers whose device memory belongs
to their own allocator under a fixed budget, and latency-critical loops.  Its
scratch lives in one static 64 MiB device array, so this test checks, through
the C ABI, that it returns what ellsolve_level_smooth returns on two calls in a
row (the second call finds the first call's leftovers in the shared array),
and that a level too large for the array is refused.  The file is collected
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("fp32,kind,n,nz", [(False, 1, 12, 16), (True, 1, 16, 16),
                                            (True, 0, 20, 12), (False, 0, 24, 8)])
def test_noalloc_smooth_matches_allocating_smoother(fp32, kind, n, nz):
    torch = _torch()
    from paper_1307_2036_gb300 import ellsolve
    sv = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.01, 1.0,
                         precision=1 if fp32 else 0)
    dt = torch.float32 if fp32 else torch.float64
    tol = 1e-6 if fp32 else 1e-12
    for call in range(2):
        shape = sv.shape(0)
        u0 = torch.tensor(inputs.uniform_pm1(shape[1:], member=200 + call), device="cuda")
        u0 = u0.expand(shape).contiguous().to(dt)
        b = torch.tensor(inputs.uniform_pm1(shape, member=300 + call) * 1e-6, device="cuda").to(dt)
        ref = u0.clone()
        sv.level_smooth(0, b, ref, nsweeps=3, rho=0.8, fp32=fp32)
        out = u0.clone()
        st = ellsolve.ellsolve_level_smooth_noalloc(sv.h, 0, int(fp32), b.data_ptr(),
                                                    out.data_ptr(), 3, 0.8)
        assert st == ellsolve.OK, ellsolve.ellsolve_last_error()
        torch.cuda.synchronize()
        err = (out - ref).double().norm() / ref.double().norm()
        assert float(err) <= tol, (call, float(err))


def test_noalloc_refuses_levels_beyond_the_static_array():
    torch = _torch()
    from paper_1307_2036_gb300 import ellsolve
    # 6 * 512^2 * 8 FP32 unknowns need ~96 MiB of scratch > 64 MiB
    sv = ellsolve.Solver(1, 512, 8, inputs.radial_levels(8), 0.01, 1.0, precision=1)
    b = torch.zeros(sv.shape(0), dtype=torch.float32, device="cuda")
    u = torch.zeros_like(b)
    st = ellsolve.ellsolve_level_smooth_noalloc(sv.h, 0, 1, b.data_ptr(), u.data_ptr(), 1, 0.8)
    assert st == ellsolve.ERR_CAPACITY
    assert b"static array" in ellsolve.ellsolve_last_error()
