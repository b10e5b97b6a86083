"""CG preconditioned by one FP64 V-cycle (opts.precond = 2, flexible beta) on
the GPU against the oracle: a fixed number of iterations with the line-Jacobi
and with the block red-black SOR V-cycle, and the converged solution."""
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

CASES = [(0, 24, 16, False, 0, 0.01, 1.0), (1, 12, 16, True, 0, 0.05, 4.0),
         (1, 16, 8, False, 1, 0.05, 0.25), (1, 64, 16, True, 0, 0.01, 1.0)]
IDS = ["box24", "sph12", "sph16e", "sph64"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def make(oracle_mod, case, smoother=0):
    kind, n, nz, graded, mapping, w2, l2 = case
    rho = 1.0 if smoother else 0.8
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
             solver=1, precond=2, smoother=smoother, damping=rho)
    # the oracle's V-cycle preconditioner with the library's options
    oracle_mod._load().og_set_mg_precond(p.og._h, 2, 2, 2, rho, 0)
    return p


@pytest.mark.parametrize("smoother", [0, 1])
@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_mg_pcg_fixed_count(torch_mod, oracle_mod, case, smoother):
    p = make(oracle_mod, case, smoother)
    f = inputs.uniform_pm1(p.og.shape(), member=401)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=4)
    u_ref, it, hist = p.og.pcg_solve(b, rtol=0.0, maxit=4)
    assert res.iterations == 4 == it
    tol = max(1e-10, fp64_tol(lambda bb: p.og.pcg_solve(bb, rtol=0.0, maxit=4)[0], b))
    assert rel_l2(p.host(x), u_ref) <= tol
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1] + 1e-13


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mg_pcg_converged(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case)
    f = inputs.uniform_pm1(p.og.shape(), member=402)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-11, maxit=60)
    u_ref = p.og.mg_solve(b, rtol=1e-13, maxit=80)[0]
    print(f"MG-PCG: {res.iterations} iterations, residual {res.rel_residual:.2e}")
    assert res.iterations <= 20
    assert rel_l2(p.host(x), u_ref) <= 1e-9
