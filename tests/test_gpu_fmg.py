"""Full multigrid (opts.fmg = 1, Sec. 4.3) on the GPU against the oracle:

  * FP64 multigrid after a fixed number of cycles, the first one full
    multigrid, element by element, on boxes and cubed spheres with 1 to 5
    levels, ragged panel sides and both prolongations;
  * CG preconditioned by one full multigrid cycle after a fixed count;
  * the mixed-precision solve (full multigrid as the first inner cycle of each
    refinement step) to the converged oracle solution, alone and as a batch of
    members with different level counts.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, mapping, omega2, lambda2
CASES = [(0, 24, 16, False, 0, 0.01, 1.0), (1, 12, 16, True, 0, 0.05, 4.0),
         (1, 16, 8, False, 1, 0.05, 0.25), (0, 40, 9, True, 0, 0.02, 2.0),
         (1, 64, 16, True, 0, 0.01, 1.0), (0, 3, 5, False, 0, 0.01, 1.0)]
IDS = ["box24", "sph12", "sph16e", "box40z9", "sph64", "box3_onelevel"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def pair(oracle_mod, case, **kw):
    kind, n, nz, graded, mapping, w2, l2 = case
    return Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
                fmg=1, **kw)


@pytest.mark.parametrize("prolong", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fmg_mg64_fixed_count(torch_mod, oracle_mod, case, prolong):
    p = pair(oracle_mod, case, prolong=prolong)
    f = inputs.uniform_pm1(p.og.shape(), member=501)
    b = p.og.volumes() * f
    for cycles in (1, 3):
        x = p.empty()
        st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=cycles)
        ref = lambda bb: p.og.mg_solve(bb, rtol=0.0, maxit=cycles, prolong_mode=prolong)[0]  # noqa
        u_ref = ref(b)
        assert res.iterations == cycles
        got = p.host(x)
        tol = max(1e-10, fp64_tol(ref, b))
        assert rel_l2(got, u_ref) <= tol, (cycles, rel_l2(got, u_ref))
        assert np.max(np.abs(got - u_ref)) <= 10 * tol * np.max(np.abs(u_ref))


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_fmg_pcg_fixed_count(torch_mod, oracle_mod, case):
    p = pair(oracle_mod, case, solver=1, precond=2)
    oracle_mod._load().og_set_mg_precond(p.og._h, 2, 2, 2, 0.8, 0)
    f = inputs.uniform_pm1(p.og.shape(), member=502)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=4)
    ref = lambda bb: p.og.pcg_solve(bb, rtol=0.0, maxit=4)[0]  # noqa: E731
    assert res.iterations == 4
    assert rel_l2(p.host(x), ref(b)) <= max(1e-10, fp64_tol(ref, b))


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fmg_mixed_precision_converged(torch_mod, oracle_mod, case):
    p = pair(oracle_mod, case, precision=1)
    f = inputs.uniform_pm1(p.og.shape(), member=503)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-10, maxit=30)
    assert st == 0 and res.rel_residual <= 1e-10
    u_ref = p.og.mg_solve(b, rtol=1e-13, maxit=80)[0]
    assert rel_l2(p.host(x), u_ref) <= 1e-9


def test_fmg_batch_mixed_levels(torch_mod, oracle_mod):
    """Members with 4, 2 and 1 levels (n 32, 8 and 3) share the launches."""
    from paper_1307_2036_gb300 import ellsolve
    pairs = [pair(oracle_mod, c, precision=1) for c in
             [(1, 32, 16, True, 0, 0.01, 1.0), (0, 8, 16, False, 0, 0.05, 4.0),
              (0, 3, 16, False, 0, 0.01, 1.0)]]
    assert sorted(p.sv.nlevels for p in pairs) == [1, 2, 4]
    fs = [inputs.uniform_pm1(p.og.shape(), member=504 + i) for i, p in enumerate(pairs)]
    xs = [p.empty() for p in pairs]
    st, out = ellsolve.solve_batch([p.sv for p in pairs], [p.dev(f) for p, f in zip(pairs, fs)],
                                   xs, rtol=1e-10, maxit=30)
    assert st == 0
    for p, f, x, res in zip(pairs, fs, xs, out):
        assert res.rel_residual <= 1e-10
        u_ref = p.og.mg_solve(p.og.volumes() * f, rtol=1e-13, maxit=80)[0]
        assert rel_l2(p.host(x), u_ref) <= 1e-9


def test_batch_rejects_mixed_fmg(torch_mod, oracle_mod):
    """Members of one batch share the launch sequence, so full multigrid is
    all or nothing."""
    from paper_1307_2036_gb300 import ellsolve
    a = pair(oracle_mod, CASES[0], precision=1)
    c = CASES[0]
    b = Pair(oracle_mod, c[0], c[1], c[2], omega2=c[5], lambda2=c[6], graded=c[3],
             mapping=c[4], precision=1, fmg=0)
    fs = [inputs.uniform_pm1(p.og.shape(), member=520 + i) for i, p in enumerate((a, b))]
    xs = [a.empty(), b.empty()]
    with pytest.raises(ellsolve.EllsolveError) as e:
        ellsolve.solve_batch([a.sv, b.sv], [a.dev(fs[0]), b.dev(fs[1])], xs, rtol=1e-8, maxit=10)
    assert e.value.status == ellsolve.ERR_ARG
