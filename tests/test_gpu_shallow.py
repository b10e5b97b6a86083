"""Shallow and very shallow multigrid (Sec. 7.3.1, Table 5) against the oracle.

The hierarchy is capped at `max_levels` levels and the coarsest level of the
cap gets `nu_coarse` undamped line sweeps (the very shallow variant of the
paper: three coarsenings and five coarsest-level sweeps).  After a fixed
number of FP64 V-cycles the library's iterate must equal the oracle's, built
with the same cap, to max(1e-10, 16x the oracle's own rounding sensitivity);
the mixed-precision solve must reach the oracle's converged solution to 1e-9.
The achieved error and the tolerance are printed.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, mapping, omega2, lambda2, max_levels, nu_coarse
CASES = [
    (0, 64, 16, True, 0, 0.01, 1.0, 4, 5),   # very shallow: 3 coarsenings (of 4), 5 coarse sweeps
    (0, 32, 16, True, 0, 0.01, 1.0, 2, 5),   # one coarsening
    (1, 32, 16, True, 0, 0.01, 1.0, 3, 5),   # sphere capped at 8 x 8 per panel
    (1, 24, 8, False, 1, 0.05, 4.0, 2, 1),   # sphere, capped, a single coarse sweep
    (0, 32, 16, True, 0, 0.01, 1.0, 0, 5),   # all levels, 5 coarsest sweeps
    (1, 16, 16, True, 0, 0.01, 1.0, 1, 3),   # one level: the V-cycle is 3 sweeps
]
IDS = ["box64-L4c5", "box32-L2c5", "sph32-L3c5", "sph24e-L2c1", "box32-c5", "sph16-L1c3"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def make(oracle_mod, case, precision):
    kind, n, nz, graded, mapping, w2, l2, maxlev, nuc = case
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
             precision=precision, max_levels=maxlev, nu_coarse=nuc)
    if maxlev:
        assert p.og.nlevels == maxlev
    return p, nuc


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_capped_vcycles_fp64_fixed_count(torch_mod, oracle_mod, case):
    p, nuc = make(oracle_mod, case, 0)
    f = inputs.uniform_pm1(p.og.shape(), member=130)
    b = p.og.volumes() * f
    ud = p.empty()
    fd = p.dev(f)
    u_ref = p.og.zeros()
    for _ in range(3):
        p.sv.vcycle(fd, ud)
        u_ref = p.og.vcycle(b, u_ref, nu_coarse=nuc)
    tol = max(1e-10, fp64_tol(
        lambda bb: p.og.mg_solve(bb, rtol=0.0, maxit=3, nu_coarse=nuc)[0], b))
    err = rel_l2(p.host(ud), u_ref)
    print(f"{case}: 3 capped V-cycles, error {err:.2e}, tolerance {tol:.2e}")
    assert err <= tol
    # the solve entry point with a fixed count: the same iterate and residual
    x = p.empty()
    st, res = p.sv.solve(fd, x, rtol=0.0, maxit=3)
    u3, it, hist = p.og.mg_solve(b, rtol=0.0, maxit=3, nu_coarse=nuc)
    assert res.iterations == it == 3
    assert rel_l2(p.host(x), u3) <= tol
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1] + 1e-15


@pytest.mark.parametrize("case", CASES[:4], ids=IDS[:4])
def test_capped_mixed_precision_solution(torch_mod, oracle_mod, case):
    p, nuc = make(oracle_mod, case, 1)
    f = inputs.uniform_pm1(p.og.shape(), member=140)
    b = p.og.volumes() * f
    u_ref, _, hist = p.og.mg_solve(b, rtol=1e-12, maxit=400, nu_coarse=nuc)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-12, maxit=400)
    err = rel_l2(p.host(x), u_ref)
    print(f"{case}: mixed {res.iterations} cycles, residual {res.rel_residual:.2e}, "
          f"error {err:.2e}")
    assert err <= 1e-9
