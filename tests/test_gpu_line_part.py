"""The partitioned line solve of the small levels (opts.line_part = 1: each
column's tridiagonal system split into eight segments, one warp each, joined by
a tridiagonal system on the seven levels between them) against the
whole-column elimination (line_part = 0) and the FP64 oracle: the same solve
up to FP32 rounding, so mixed-precision solves take the same number of
V-cycles and reach the same solution."""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, omega2, lambda2, smoother
# (sizes that the oracle's FP64 multigrid solves to 1e-12 in seconds)
CASES = [(1, 24, 128, True, 0.01, 1.0, 0), (0, 64, 64, True, 0.1, 25.0, 0),
         (1, 16, 256, True, 0.05, 4.0, 1), (1, 24, 16, False, 0.01, 1.0, 0)]
IDS = ["sph24z128", "box64z64strong", "sph16z256rb", "sph24z16"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_partitioned_and_whole_column_solves_agree(torch_mod, oracle_mod, case):
    kind, n, nz, graded, w2, l2, smoother = case
    out = {}
    for line_part in (1, 0):
        p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, precision=1,
                 smoother=smoother, line_part=line_part)
        f = inputs.uniform_pm1(p.og.shape(), member=701)
        x = p.empty()
        st, res = p.sv.solve(p.dev(f), x, rtol=1e-10, maxit=60)
        out[line_part] = (st, res.iterations, p.host(x))
    u_ref = p.og.mg_solve(p.og.volumes() * f, rtol=1e-12, maxit=100)[0]
    e1, e0 = rel_l2(out[1][2], u_ref), rel_l2(out[0][2], u_ref)
    print(f"{(kind, n, nz, smoother)}: partitioned {out[1][1]} V-cycles (error {e1:.2e}), "
          f"whole column {out[0][1]} (error {e0:.2e})")
    # the same outcome (strongly coupled columns stop at the FP64 floor,
    # NOT_CONVERGED, in both) after the same number of V-cycles
    assert out[1][0] == out[0][0]
    assert abs(out[1][1] - out[0][1]) <= 1
    assert e1 <= 1e-9 and e0 <= 1e-9
