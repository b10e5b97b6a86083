"""Vertical background profiles (ellsolve_create_profiles) on the GPU against
the oracle with the same profiles: the operator, the FP32 kernels, fixed
numbers of V-cycles and CG iterations, and the mixed-precision solution."""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import fp64_tol, rel_l2, require_gpu
from test_oracle_profiles import profiles

pytestmark = pytest.mark.gpu

CASES = [(0, 24, 16, True, 0.01, 1.0), (1, 12, 16, True, 0.05, 4.0), (1, 64, 16, True, 0.01, 1.0)]
IDS = ["box24", "sph12", "sph64"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


class PPair:
    def __init__(self, oracle_mod, case, **opts):
        import torch
        from paper_1307_2036_gb300 import ellsolve
        kind, n, nz, graded, w2, l2 = case
        self.torch = torch
        self.r = inputs.radial_levels(nz, graded=graded)
        self.pc, self.qf = profiles(nz, self.r)
        self.og = oracle_mod.Grid(kind, n, nz, self.r, w2, l2, p_cell=self.pc, q_face=self.qf,
                                  precond=opts.get("precond", 0))
        self.sv = ellsolve.Solver(kind, n, nz, self.r, w2, l2, p_cell=self.pc, q_face=self.qf,
                                  **opts)

    def dev(self, a, fp32=False):
        t = self.torch.tensor(np.ascontiguousarray(a), dtype=self.torch.float64, device="cuda")
        return t.float().contiguous() if fp32 else t

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.double().cpu().numpy()

    def empty(self, lev=0, fp32=False):
        dt = self.torch.float32 if fp32 else self.torch.float64
        return self.torch.zeros(self.og.shape(lev), dtype=dt, device="cuda")


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_profiles_operator_and_vcycles_fp64(torch_mod, oracle_mod, case):
    p = PPair(oracle_mod, case)
    u = inputs.uniform_pm1(p.og.shape(), member=301)
    y = p.empty()
    p.sv.apply(p.dev(u), y)
    assert rel_l2(p.host(y), p.og.apply(u)) <= 1e-13
    f = inputs.uniform_pm1(p.og.shape(), member=302)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=3)
    u3, it, hist = p.og.mg_solve(b, rtol=0.0, maxit=3)
    tol = max(1e-10, fp64_tol(lambda bb: p.og.mg_solve(bb, rtol=0.0, maxit=3)[0], b))
    assert res.iterations == 3 == it
    assert rel_l2(p.host(x), u3) <= tol


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_profiles_fp32_smoother_and_mixed_solution(torch_mod, oracle_mod, case):
    p = PPair(oracle_mod, case, precision=1)
    b = p.og.volumes() * inputs.uniform_pm1(p.og.shape(), member=303)
    b = b.astype(np.float32).astype(np.float64)
    uh = np.broadcast_to(inputs.uniform_pm1(p.og.shape()[1:], member=304), p.og.shape())
    uh = uh.astype(np.float32).astype(np.float64)
    ud = p.dev(uh, True)
    p.sv.level_smooth(0, p.dev(b, True), ud, nsweeps=2, rho=0.8, fp32=True)
    assert rel_l2(p.host(ud), p.og.smooth(b, uh, 2, 0.8, 0)) <= 1e-5
    f = inputs.uniform_pm1(p.og.shape(), member=305)
    u_ref = p.og.mg_solve(p.og.volumes() * f, rtol=1e-13, maxit=80)[0]
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-12, maxit=80)
    assert rel_l2(p.host(x), u_ref) <= 1e-9


@pytest.mark.parametrize("precond", [0, 1])
def test_profiles_pcg_fixed_count(torch_mod, oracle_mod, precond):
    p = PPair(oracle_mod, CASES[1], solver=1, precond=precond)
    f = inputs.uniform_pm1(p.og.shape(), member=306)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=15)
    u_ref, it, hist = p.og.pcg_solve(b, rtol=0.0, maxit=15)
    tol = max(1e-10, fp64_tol(lambda bb: p.og.pcg_solve(bb, rtol=0.0, maxit=15)[0], b))
    assert res.iterations == 15 == it
    assert rel_l2(p.host(x), u_ref) <= tol


def test_profiles_rejected_when_not_positive(torch_mod):
    from paper_1307_2036_gb300 import ellsolve
    r = inputs.radial_levels(8)
    for pc, qf in ((np.full(8, -1.0), None), (None, np.zeros(9))):
        with pytest.raises(ellsolve.EllsolveError) as e:
            ellsolve.Solver(1, 8, 8, r, 0.01, 1.0, p_cell=pc, q_face=qf)
        assert e.value.status == ellsolve.ERR_ARG
