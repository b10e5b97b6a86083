"""Edge cases of the library against the oracle: degenerate grids (one cell
per panel, a single level, a single vertical level, a column longer than the
smoother's staged blocks), an all-zero right-hand side, a zero iteration
budget and invalid arguments rejected on the host."""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, omega2, lambda2, coarsest_min
EDGE = [
    (1, 1, 1, False, 0.01, 1.0, 4),     # 6 unknowns, one level, one vertical level
    (1, 1, 9, True, 0.01, 1.0, 4),      # one cell per panel, a 9-level column
    (0, 3, 5, False, 0.01, 1.0, 1),     # odd n: the coarsest level is the finest
    (1, 8, 1, False, 0.01, 1.0, 1),     # nz = 1: no vertical coupling, 4 levels (8..1)
    (0, 4, 1001, True, 0.01, 1.0, 1),   # a long, graded column, nz not a multiple of 8
    (1, 6, 13, True, 0.01, 1.0, 1),     # n = 6 -> 3: the cube's 6 x 3 x 3 coarsest level
]
EIDS = ["sph1z1", "sph1z9", "box3", "sph8z1", "box4z1001", "sph6z13"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def pair(oracle_mod, case, **kw):
    kind, n, nz, graded, w2, l2, cmin = case
    return Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded,
                coarsest_min=cmin, **kw)


@pytest.mark.parametrize("case", EDGE, ids=EIDS)
def test_edge_operator_and_smoother(torch_mod, oracle_mod, case):
    p = pair(oracle_mod, case)
    u = inputs.uniform_pm1(p.og.shape(), member=61)
    b = p.og.volumes() * inputs.uniform_pm1(p.og.shape(), member=62)
    y = p.empty()
    p.sv.apply(p.dev(u), y)
    assert rel_l2(p.host(y), p.og.apply(u)) <= 1e-13
    for lev in range(p.og.nlevels):
        ul = inputs.uniform_pm1(p.og.shape(lev), member=63 + lev)
        bl = p.og.volumes(lev) * inputs.uniform_pm1(p.og.shape(lev), member=73 + lev)
        ud = p.dev(ul)
        p.sv.level_smooth(lev, p.dev(bl), ud, nsweeps=2, rho=0.8)
        ref = p.og.smooth(bl, ul, nsweeps=2, rho=0.8, lev=lev)
        tol = fp64_tol(lambda bb, uu: p.og.smooth(bb, uu, 2, 0.8, lev), bl, ul)
        assert rel_l2(p.host(ud), ref) <= tol, lev


@pytest.mark.parametrize("case", EDGE, ids=EIDS)
def test_edge_solves_match_dense_or_oracle(torch_mod, oracle_mod, case):
    p64 = pair(oracle_mod, case)
    f = inputs.uniform_pm1(p64.og.shape(), member=80)
    b = p64.og.volumes() * f
    # fixed count: same iterate as the oracle's V-cycles
    x = p64.empty()
    st, res = p64.sv.solve(p64.dev(f), x, rtol=0.0, maxit=3)
    u3, it, hist = p64.og.mg_solve(b, rtol=0.0, maxit=3)
    assert res.iterations == 3 == it
    tol = max(1e-10, fp64_tol(lambda bb: p64.og.mg_solve(bb, rtol=0.0, maxit=3)[0], b))
    assert rel_l2(p64.host(x), u3) <= tol
    # converged, mixed precision: against the exact discrete solution where the
    # dense matrix is small, else against the oracle's multigrid solution at its
    # FP64 floor, within 16x that solution's own rounding sensitivity
    pm = pair(oracle_mod, case, precision=1)
    xm = pm.empty()
    st, res = pm.sv.solve(pm.dev(f), xm, rtol=1e-12, maxit=400)
    # the attainable FP64 residual: the oracle's smallest over 30 V-cycles (on a
    # long graded column it is ~5e-9, the rounding floor eps |A| |u| / |b|)
    u30, _, hist30 = p64.og.mg_solve(b, rtol=0.0, maxit=30)
    floor = float(np.min(hist30))
    assert st in (0, 1) and res.rel_residual <= max(1e-11, 4 * floor)
    N = int(np.prod(p64.og.shape()))
    if N <= 4000:
        exact = np.linalg.solve(p64.og.dense(), b.reshape(-1)).reshape(p64.og.shape())
        tol = 1e-9
    else:
        exact = u30
        tol = max(1e-9, fp64_tol(lambda bb: p64.og.mg_solve(bb, rtol=0.0, maxit=30)[0], b))
    err = rel_l2(pm.host(xm), exact)
    print(f"mixed: {res.iterations} cycles, residual {res.rel_residual:.2e}, error {err:.2e}, tol {tol:.2e}")
    assert err <= tol


@pytest.mark.parametrize("precision,solver", [(0, 0), (1, 0), (0, 1)])
def test_zero_rhs_and_zero_budget(torch_mod, oracle_mod, precision, solver):
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    p = pair(oracle_mod, (1, 8, 16, True, 0.01, 1.0, 4), precision=precision, solver=solver)
    x = torch.full(p.og.shape(), 3.0, dtype=torch.float64, device="cuda")
    st, res = p.sv.solve(p.empty(), x, rtol=1e-8, maxit=20)
    torch.cuda.synchronize()
    assert st == ellsolve.OK and res.iterations == 0 and res.rel_residual == 0.0
    assert torch.count_nonzero(x).item() == 0
    f = inputs.uniform_pm1(p.og.shape(), member=90)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-8, maxit=0)
    torch.cuda.synchronize()
    assert st == ellsolve.NOT_CONVERGED and res.iterations == 0 and res.rel_residual == 1.0
    assert torch.count_nonzero(x).item() == 0


def test_invalid_arguments_rejected(torch_mod):
    from paper_1307_2036_gb300 import ellsolve
    r = inputs.radial_levels(8)
    bad = [
        dict(kind=1, n=0, nz=8, r_levels=r),
        dict(kind=1, n=8, nz=0, r_levels=r[:1]),
        dict(kind=2, n=8, nz=8, r_levels=r),
        dict(kind=1, n=8, nz=8, r_levels=r[::-1].copy()),
        dict(kind=1, n=8, nz=8, r_levels=r, omega2=0.0),
        dict(kind=1, n=8, nz=8, r_levels=r, solver=1, precision=1),
        dict(kind=1, n=8, nz=8, r_levels=r, damping=2.5),
        dict(kind=1, n=8, nz=8, r_levels=r, smoother=2),
        dict(kind=1, n=8, nz=8, r_levels=r, solver=1, precond=3),
        dict(kind=1, n=8, nz=8, r_levels=r, fmg=2),
        dict(kind=1, n=8, nz=8, r_levels=r, precision=1, refine=2),
    ]
    for kw in bad:
        args = dict(omega2=0.01, lambda2=1.0)
        args.update(kw)
        with pytest.raises(ellsolve.EllsolveError) as e:
            ellsolve.Solver(args.pop("kind"), args.pop("n"), args.pop("nz"), args.pop("r_levels"),
                            args.pop("omega2"), args.pop("lambda2"), **args)
        assert e.value.status == ellsolve.ERR_ARG, kw
