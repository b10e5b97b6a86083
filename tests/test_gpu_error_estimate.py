"""The per-result error estimate of the mixed-precision solver against the true
error: ||x - x*|| / ||x*||, with x* the oracle's FP64 multigrid solution
iterated to its attainable residual.

The estimate is q / (1 - q) ||dx_last|| / ||dx_first|| from the refinement
updates (the error left by a linearly contracting iteration), q the last
step's residual reduction scaled by the ratio of error to residual
contraction of the step before.  Measured, the estimate lies within a factor
0.23 .. 12 of the true error over these cases: two-step solves (rtol 1e-4 /
1e-6) underestimate by up to 4.3x, their second step contracting the error
less than anything measured before it shows; later steps are within 2.3x
except at the FP64 floor.  The bar is a factor 8 below and 50 above (or an
estimate under 1e-12 when the true error is at the FP64 floor); the FP64
solvers report -1.  The ratio estimate / error is printed for every case.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

CASES = [  # kind, n, nz, graded, omega2, lambda2
    (0, 32, 32, False, 0.01, 1.0),
    (0, 64, 32, True, 0.05, 4.0),
    (1, 16, 32, True, 0.01, 1.0),
    (1, 24, 64, True, 0.002, 0.25),
]
IDS = ["box32", "box64g", "sph16", "sph24"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_error_estimate_tracks_the_true_error(torch_mod, oracle_mod, case):
    kind, n, nz, graded, w2, l2 = case
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, precision=1)
    f = inputs.uniform_pm1(p.og.shape(), member=150)
    b = p.og.volumes() * f
    x_star, _, _ = p.og.mg_solve(b, rtol=1e-13, maxit=200)
    for rtol in (1e-4, 1e-6, 1e-8, 1e-10):
        x = p.empty()
        st, res = p.sv.solve(p.dev(f), x, rtol=rtol, maxit=80)
        err = rel_l2(p.host(x), x_star)
        est = res.rel_error_est
        print(f"{case} rtol {rtol:g}: {res.iterations} V-cycles, residual {res.rel_residual:.2e}, "
              f"error {err:.2e}, estimate {est:.2e}, ratio {est / max(err, 1e-300):.2f}")
        assert est >= 0.0
        assert est >= err / 8.0
        assert est <= 50.0 * err or est <= 1e-12


def test_fp64_solvers_report_no_estimate(torch_mod, oracle_mod):
    for solver in (0, 1):
        p = Pair(oracle_mod, 0, 16, 16, precision=0, solver=solver)
        f = inputs.uniform_pm1(p.og.shape(), member=151)
        x = p.empty()
        st, res = p.sv.solve(p.dev(f), x, rtol=1e-6, maxit=100)
        assert res.rel_error_est == -1.0
