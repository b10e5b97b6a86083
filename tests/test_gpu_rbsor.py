"""Block red-black SOR line smoother and block red-black SSOR CG
preconditioner (Eq. BlockRBSOR; Sec. 6.2.1 colouring; Sec. 7.2) on the GPU,
through the C ABI, against the oracle on the same seeded inputs.

Tolerances as in test_gpu_parity.py: FP64 within 16x the oracle's own
rounding sensitivity (at least 1e-13, and 1e-10 after iterations); FP32
sweeps 1e-5 relative L2 and 2e-5 of the largest value element by element;
mixed-precision solutions 1e-9.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, mapping, omega2, lambda2
CASES = [
    (0, 24, 16, False, 0, 0.01, 1.0),    # box: an exact two-colouring
    (1, 12, 16, True, 0, 0.01, 1.0),     # sphere: same-colour neighbours across some edges
    (1, 16, 8, False, 1, 0.05, 0.25),    # equidistant sphere
    (0, 128, 16, True, 0, 0.02, 4.0),    # box, levels with n % 32 == 0 (aligned FP32 kernel)
    (1, 64, 16, True, 0, 0.01, 1.0),     # sphere, aligned levels
]
IDS = ["box24", "sph12", "sph16e", "box128", "sph64"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def make(oracle_mod, case, **kw):
    kind, n, nz, graded, mapping, w2, l2 = case
    return Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
                smoother=1, **kw)


def rand(shape, member):
    return inputs.uniform_pm1(shape, member=member)


def f32exact(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
@pytest.mark.parametrize("nsweeps,rho", [(1, 1.0), (2, 1.2)])
def test_rb_smoother_fp64(torch_mod, oracle_mod, case, nsweeps, rho):
    p = make(oracle_mod, case)
    for lev in range(p.og.nlevels):
        u = rand(p.og.shape(lev), 220 + lev)
        b = p.og.volumes(lev) * rand(p.og.shape(lev), 230 + lev)
        ud = p.dev(u)
        p.sv.level_smooth(lev, p.dev(b), ud, nsweeps=nsweeps, rho=rho)
        ref = p.og.smooth(b, u, nsweeps=nsweeps, rho=rho, lev=lev)
        tol = fp64_tol(lambda bb, uu: p.og.smooth(bb, uu, nsweeps, rho, lev), b, u)
        assert rel_l2(p.host(ud), ref) <= tol, lev


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rb_smoother_fp32(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, precision=1)
    for lev in range(min(3, p.og.nlevels)):
        b = f32exact(p.og.volumes(lev) * rand(p.og.shape(lev), 240 + lev))
        # constant in k (see test_kernels_fp32): no large vertical differences
        uh = f32exact(np.broadcast_to(rand(p.og.shape(lev)[1:], 245 + lev), p.og.shape(lev)))
        ud = p.dev(uh, True)
        p.sv.level_smooth(lev, p.dev(b, True), ud, nsweeps=2, rho=1.0, fp32=True)
        ref = p.og.smooth(b, uh, 2, 1.0, lev)
        got = p.host(ud)
        assert rel_l2(got, ref) <= 1e-5, lev
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)), lev


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_rb_vcycles_fp64_fixed_count(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, damping=1.0)
    f = rand(p.og.shape(), 250)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=3)
    u3, it, hist = p.og.mg_solve(b, rtol=0.0, maxit=3, rho=1.0)
    assert res.iterations == 3 == it
    tol = max(1e-10, fp64_tol(lambda bb: p.og.mg_solve(bb, rtol=0.0, maxit=3, rho=1.0)[0], b))
    assert rel_l2(p.host(x), u3) <= tol
    # (near the FP64 floor the two residual norms differ by rounding alone)
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1] + 1e-13


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_rb_mixed_precision_solution(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, precision=1, damping=1.0)
    f = rand(p.og.shape(), 260)
    b = p.og.volumes() * f
    u_ref, it_ref, hist_ref = p.og.mg_solve(b, rtol=1e-13, maxit=80, rho=1.0)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-12, maxit=80)
    err = rel_l2(p.host(x), u_ref)
    print(f"RB-SOR mixed: {res.iterations} cycles (oracle FP64 {it_ref}), error {err:.2e}")
    assert err <= 1e-9


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_pcg_rb_ssor_fixed_count(torch_mod, oracle_mod, case):
    kind, n, nz, graded, mapping, w2, l2 = case
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
             solver=1, precond=1)
    f = rand(p.og.shape(), 270)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=12)
    u_ref, it, hist = p.og.pcg_solve(b, rtol=0.0, maxit=12)
    assert res.iterations == 12 == it
    tol = max(1e-10, fp64_tol(lambda bb: p.og.pcg_solve(bb, rtol=0.0, maxit=12)[0], b))
    assert rel_l2(p.host(x), u_ref) <= tol
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1]


def test_rb_batch_equals_alone(torch_mod, oracle_mod):
    """Red-black and Jacobi members in one batch give the bits they give alone."""
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    specs = [(1, 8, 16, 1), (0, 24, 12, 0), (1, 32, 32, 1), (0, 64, 16, 1), (1, 12, 8, 0)]
    solvers, rhs = [], []
    for m, (kind, n, nz, sm) in enumerate(specs):
        s = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.01, 1.0,
                            precision=1, smoother=sm, damping=1.0 if sm else 0.8)
        solvers.append(s)
        rhs.append(torch.tensor(inputs.uniform_pm1(s.shape(), member=m), device="cuda"))
    alone = []
    for s, f in zip(solvers, rhs):
        x = torch.zeros_like(f)
        st, res = s.solve(f, x, rtol=1e-8, maxit=30)
        alone.append((x.clone(), res.iterations))
    xs = [torch.zeros_like(f) for f in rhs]
    st, res = ellsolve.solve_batch(solvers, rhs, xs, rtol=1e-8, maxit=30)
    for (xa, ita), xb, rb in zip(alone, xs, res):
        assert ita == rb.iterations
        assert torch.equal(xa, xb)
        assert rb.rel_residual <= 1e-8
