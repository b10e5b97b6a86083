"""The allocation-free line-smoothing entry point against the allocating one.

ellsolve_level_smooth_noalloc exists for callers that cannot call cudaMalloc:
host programs whose device memory belongs to their own allocator or pool under
a fixed budget, and latency-critical loops where a cudaMalloc / cudaFree pair
could synchronise the device.  Its scratch lives in one static 64 MiB device
array.  This test checks, through the C ABI, that it returns exactly what
ellsolve_level_smooth returns (the same kernels over the same work items) on
two calls in a row -- the second call finds the first call's leftovers in the
shared array -- that the free device memory does not change across a call,
and that a level too large for the array is refused.  The cases cover line
Jacobi and block red-black SOR in FP64 and FP32, including an FP32 level large
enough for the twisted smoother to park its eliminated right-hand side in
tensor memory.  The file is collected last so that a run stopping at the first
failure has run every other test.
"""
import pytest

from paper_1307_2036_gb300 import inputs

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


CASES = [
    # (fp32, kind, n, nz, smoother)
    (False, 1, 12, 16, 0),
    (True, 1, 16, 16, 0),
    (True, 0, 20, 12, 0),
    (False, 0, 24, 8, 0),
    (False, 1, 12, 16, 1),
    (True, 1, 16, 16, 1),
    # 6 x 64^2 columns = 192 blocks of 128: the twisted smoother with f' in TMEM
    (True, 1, 64, 128, 0),
    (True, 1, 64, 128, 1),
]


@pytest.mark.parametrize("fp32,kind,n,nz,smoother", CASES)
def test_noalloc_smooth_matches_allocating_smoother(fp32, kind, n, nz, smoother):
    torch = _torch()
    from paper_1307_2036_gb300 import ellsolve
    sv = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.01, 1.0,
                         precision=1 if fp32 else 0, smoother=smoother)
    dt = torch.float32 if fp32 else torch.float64
    shape = sv.shape(0)
    for call in range(2):
        u0 = torch.tensor(inputs.uniform_pm1(shape, member=200 + call), device="cuda").to(dt)
        b = torch.tensor(inputs.uniform_pm1(shape, member=300 + call) * 1e-6,
                         device="cuda").to(dt)
        ref = u0.clone()
        sv.level_smooth(0, b, ref, nsweeps=3, rho=0.8, fp32=fp32)
        out = u0.clone()
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = ellsolve.ellsolve_level_smooth_noalloc(sv.h, 0, int(fp32), b.data_ptr(),
                                                    out.data_ptr(), 3, 0.8)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        assert st == ellsolve.OK, ellsolve.ellsolve_last_error()
        assert torch.equal(out, ref), (call, float((out - ref).abs().max()))
        # the first call of the process may load the module (and its static
        # array); from then on a call allocates nothing
        if call == 1:
            assert free_after == free_before, (free_before, free_after)


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
