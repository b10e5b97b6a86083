"""The refinement residual of the mixed-precision solve (opts.refine): tracked
(double-float update r <- r - A e with a rounding bound, FP64 recomputation
when the bound is not small) against recomputed in FP64 at every step.  The
oracle's FP64 residual of the returned x is the reference for the reported
residual; its multigrid solution for x."""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, mapping, omega2, lambda2
CASES = [(0, 32, 16, True, 0, 0.01, 1.0), (1, 16, 32, True, 0, 0.05, 4.0),
         (1, 24, 16, False, 1, 0.01, 0.25), (0, 64, 64, True, 0, 0.1, 100.0)]
IDS = ["box32", "sph16", "sph24e", "box64_strong"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def pair(oracle_mod, case, **kw):
    kind, n, nz, graded, mapping, w2, l2 = case
    return Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
                precision=1, **kw)


def true_rel(p, f, x):
    b = p.og.volumes() * f
    return np.linalg.norm(p.og.residual(b, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_first_step_identical_and_tracked_residual_exact(torch_mod, oracle_mod, case):
    pt, pf = pair(oracle_mod, case, refine=0), pair(oracle_mod, case, refine=1)
    f = inputs.uniform_pm1(pt.og.shape(), member=601)
    inner = 3
    xs = {}
    for name, p in (("t", pt), ("f", pf)):
        for steps in (1, 2):
            x = p.empty()
            st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=inner * steps)
            xs[name, steps] = (p.host(x), res.rel_residual)
    # one step: the same inner right-hand side, so the same x
    assert np.array_equal(xs["t", 1][0], xs["f", 1][0])
    # the tracked residual after two steps is the true residual of the x returned
    for steps in (1, 2):
        xt, rep = xs["t", steps]
        rel = true_rel(pt, f, xt)
        assert abs(rep - rel) <= 1e-6 * rel + 1e-15, (steps, rep, rel)
    # and the two modes' iterates agree to the accuracy of the inner solve
    assert rel_l2(xs["t", 2][0], xs["f", 2][0]) <= 1e-5


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_converged_solution_and_reported_residual(torch_mod, oracle_mod, case, refine):
    p = pair(oracle_mod, case, refine=refine)
    f = inputs.uniform_pm1(p.og.shape(), member=602)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-10, maxit=60)
    xh = p.host(x)
    rel = true_rel(p, f, xh)
    u_ref = p.og.mg_solve(p.og.volumes() * f, rtol=1e-13, maxit=100)[0]
    print(f"refine {refine}: status {st}, {res.iterations} cycles, reported "
          f"{res.rel_residual:.3e}, true {rel:.3e}")
    assert abs(res.rel_residual - rel) <= 1e-2 * rel + 1e-16
    if st == 0:
        assert rel <= 1.02e-10
        assert rel_l2(xh, u_ref) <= 1e-9


def test_tight_tolerance_falls_back_to_fp64(torch_mod, oracle_mod):
    """At rtol 1e-13 the tracked bound cannot certify the residual: the solve
    recomputes it in FP64 and reports the true residual of its x."""
    p = pair(oracle_mod, CASES[1], refine=0)
    f = inputs.uniform_pm1(p.og.shape(), member=603)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-13, maxit=60)
    rel = true_rel(p, f, p.host(x))
    assert abs(res.rel_residual - rel) <= 1e-2 * rel + 1e-16


def test_batch_mixed_modes_equal_alone(torch_mod, oracle_mod):
    from paper_1307_2036_gb300 import ellsolve
    ps = [pair(oracle_mod, CASES[0], refine=0), pair(oracle_mod, CASES[1], refine=1),
          pair(oracle_mod, CASES[2], refine=0)]
    fs = [inputs.uniform_pm1(p.og.shape(), member=610 + i) for i, p in enumerate(ps)]
    alone = []
    for p, f in zip(ps, fs):
        x = p.empty()
        st, res = p.sv.solve(p.dev(f), x, rtol=1e-9, maxit=40)
        alone.append((p.host(x), res.rel_residual, res.iterations))
    xs = [p.empty() for p in ps]
    st, out = ellsolve.solve_batch([p.sv for p in ps], [p.dev(f) for p, f in zip(ps, fs)], xs,
                                   rtol=1e-9, maxit=40)
    for p, x, res, (xa, ra, ia) in zip(ps, xs, out, alone):
        assert np.array_equal(p.host(x), xa)
        assert res.rel_residual == ra and res.iterations == ia


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("case", CASES[:2], ids=IDS[:2])
def test_power_of_two_rhs_scales_the_result_exactly(torch_mod, oracle_mod, case, refine):
    """x(2^k f) = 2^k x(f) bit for bit, with the same V-cycle count and relative
    residual: the refinement scales are powers of two.  From x = 0 the first
    scale normalises b for f = 1; for |k| beyond 2^20 of that (k = +-24, +-40)
    b is formed again with its own scale, and the result is still the same."""
    torch = torch_mod
    p = pair(oracle_mod, case, refine=refine)
    f = torch.tensor(inputs.uniform_pm1(p.og.shape(), member=604), device="cuda")
    runs = {}
    for k in (0, 3, -11, 24, -24, 40, -40):
        x = torch.empty_like(f)
        st, res = p.sv.solve(f * 2.0 ** k, x, rtol=1e-9, maxit=40)
        torch.cuda.synchronize()
        runs[k] = (st, res.iterations, res.rel_residual, x)
    st0, it0, rel0, x0 = runs[0]
    for k, (st, it, rel, x) in runs.items():
        print(f"k {k:+d}: status {st}, {it} V-cycles, residual {rel:.3e}")
        assert (st, it, rel) == (st0, it0, rel0), k
        assert torch.equal(x, x0 * 2.0 ** k), k
