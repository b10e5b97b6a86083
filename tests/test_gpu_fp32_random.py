"""FP32 line smoother on fully random iterates at n_z = 128, on the launches that
park the eliminated right-hand side in tensor memory (at least 152 blocks of
128 columns), against the FP64 oracle element by element.

An FP32 sweep rounds the residual b - A u, whose terms are much larger than
the residual itself on graded columns, and the tridiagonal solve amplifies that
rounding by the column's condition.  The tolerance is therefore derived, not
fixed: 16x the oracle's own response to binary32-level (4 eps32) relative
changes of its inputs u and b (an empirical condition estimate at FP32
precision), in the relative L2 norm and, element by element, relative to the
largest element.  The achieved error and the tolerance are printed.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp32_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, omega2, lambda2, smoother
CASES = [
    (1, 64, 128, True, 0.01, 1.0, 0),    # 192 blocks, n % 32 == 0 (aligned staging)
    (1, 80, 128, True, 0.01, 1.0, 0),    # 300 blocks, n % 32 != 0 (neighbour buffer)
    (1, 64, 128, True, 0.01, 1.0, 1),    # block red-black SOR half-sweeps
    (0, 160, 128, True, 0.1, 25.0, 0),   # box, strong vertical coupling (ill-conditioned columns)
]
IDS = ["sph64z128", "sph80z128", "sph64z128rb", "box160z128strong"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def f32exact(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp32_smoother_random_iterate(torch_mod, oracle_mod, case):
    kind, n, nz, graded, w2, l2, smoother = case
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, precision=1,
             smoother=smoother)
    ncol = p.og.ncol()
    assert (ncol + 127) // 128 >= 152  # the tensor-memory launch
    sh = p.og.shape()
    u = f32exact(inputs.uniform_pm1(sh, member=501))
    b = f32exact(p.og.volumes() * inputs.uniform_pm1(sh, member=502))
    rho = 1.0 if smoother == 1 else 0.8
    fn = lambda bb, uu: p.og.smooth(bb, uu, 2, rho) if smoother == 0 else _rb(p, bb, uu, rho)
    ref = fn(b, u)
    tol_l2 = fp32_tol(fn, b, u)
    tol_max = fp32_tol(fn, b, u, norm="max")
    ud = p.dev(u, True)
    p.sv.level_smooth(0, p.dev(b, True), ud, nsweeps=2, rho=rho, fp32=True)
    got = p.host(ud)
    err = rel_l2(got, ref)
    emax = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"{n}x{n}x{nz} smoother {smoother}: L2 {err:.2e} (tol {tol_l2:.2e}), "
          f"max {emax:.2e} (tol {tol_max:.2e})")
    assert err <= tol_l2
    assert emax <= tol_max


def _rb(p, b, u, rho):
    """Two block red-black SOR sweeps of the oracle (smoother 1)."""
    og = p.og
    from oracle import Grid
    g = Grid(og.kind, og.n, og.nz, p.r, og.omega2, og.lambda2, smoother=1)
    return g.smooth(b, u, 2, rho)
