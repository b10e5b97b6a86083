"""GPU parity: the CUDA library against the FP64 oracle, element by element, on
the same seeded inputs, through the C ABI (ctypes binding).

Tolerances:
  FP64 kernels         relative L2 1e-13 where no solve is involved (stencil,
                       transfers); where a tridiagonal solve or an iteration
                       amplifies rounding, 16x the oracle's own sensitivity to
                       eps-level perturbations of its inputs, at least 1e-13;
                       after a fixed number of V-cycles / CG iterations,
                       max(1e-10, that sensitivity bound).
  FP32 kernels         relative L2 1e-5 against the FP64 oracle on inputs that
                       are exactly representable in FP32 (rounding of one pass).
  mixed-precision      relative L2 1e-9 against the oracle's converged solution.
Sizes span several 128-column tiles with a ragged last tile.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import Pair, fp64_tol, rel_l2, require_gpu, sensitivity

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, mapping, omega2, lambda2
CASES = [
    (0, 24, 16, False, 0, 0.01, 1.0),    # box, 576 columns, 3 levels
    (0, 20, 12, True, 0, 0.1, 25.0),     # box, graded, strong coupling
    (1, 12, 16, True, 0, 0.01, 1.0),     # equiangular sphere, 864 columns
    (1, 16, 8, False, 1, 0.05, 0.25),    # equidistant sphere, 3 levels
    (1, 8, 128, True, 0, 0.01, 1.0),     # the 128-level graded column of the sphere configs
    (0, 12, 19, True, 0, 0.02, 4.0),     # n_z = 19: small levels split into 10 + 9 levels
]
IDS = ["box24", "box20g", "sph12", "sph16e", "sph8z128", "box12z19"]


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def make(oracle_mod, case, precision=0, **kw):
    kind, n, nz, graded, mapping, w2, l2 = case
    return Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, mapping=mapping,
                precision=precision, **kw)


def rand(shape, member, scale=1.0):
    return scale * inputs.uniform_pm1(shape, member=member)


def f32exact(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_apply_and_residual_fp64(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case)
    u = rand(p.og.shape(), 1)
    b = p.og.volumes() * rand(p.og.shape(), 2)
    y = p.empty()
    p.sv.apply(p.dev(u), y)
    assert rel_l2(p.host(y), p.og.apply(u)) <= 1e-13
    for lev in range(p.og.nlevels):
        ul = rand(p.og.shape(lev), 3 + lev)
        bl = p.og.volumes(lev) * rand(p.og.shape(lev), 10 + lev)
        r = p.empty(lev)
        p.sv.level_residual(lev, p.dev(bl), p.dev(ul), r)
        assert rel_l2(p.host(r), p.og.residual(bl, ul, lev)) <= 1e-13, lev


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("nsweeps", [1, 3])
def test_line_smoother_fp64(torch_mod, oracle_mod, case, nsweeps):
    p = make(oracle_mod, case)
    for lev in range(p.og.nlevels):
        u = rand(p.og.shape(lev), 20 + lev)
        b = p.og.volumes(lev) * rand(p.og.shape(lev), 30 + lev)
        ud = p.dev(u)
        p.sv.level_smooth(lev, p.dev(b), ud, nsweeps=nsweeps, rho=0.8)
        ref = p.og.smooth(b, u, nsweeps=nsweeps, rho=0.8, lev=lev)
        tol = fp64_tol(lambda bb, uu: p.og.smooth(bb, uu, nsweeps, 0.8, lev), b, u)
        err = rel_l2(p.host(ud), ref)
        print(f"smooth lev {lev}: err {err:.2e} tol {tol:.2e}")
        assert err <= tol, lev


@pytest.mark.parametrize("case", CASES, ids=IDS)
@pytest.mark.parametrize("mode", [0, 1])
def test_transfers_fp64(torch_mod, oracle_mod, case, mode):
    p = make(oracle_mod, case, prolong=mode)
    for lev in range(p.og.nlevels - 1):
        u = rand(p.og.shape(lev), 40 + lev)
        b = p.og.volumes(lev) * rand(p.og.shape(lev), 50 + lev)
        bc = p.empty(lev + 1)
        p.sv.level_restrict_residual(lev, p.dev(b), p.dev(u), bc)
        ref = p.og.restrict(p.og.residual(b, u, lev), lev)
        assert rel_l2(p.host(bc), ref) <= 1e-13
        uc = rand(p.og.shape(lev + 1), 60 + lev)
        uf = p.dev(u)
        p.sv.level_prolong_add(lev, p.dev(uc), uf)
        assert rel_l2(p.host(uf), p.og.prolong_add(uc, u, lev, mode=mode)) <= 1e-15


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_kernels_fp32(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, precision=1)
    for lev in range(p.og.nlevels):
        u = f32exact(rand(p.og.shape(lev), 70 + lev))
        b = f32exact(p.og.volumes(lev) * rand(p.og.shape(lev), 80 + lev))
        r = p.empty(lev, fp32=True)
        p.sv.level_residual(lev, p.dev(b, True), p.dev(u, True), r, fp32=True)
        assert rel_l2(p.host(r), p.og.residual(b, u, lev)) <= 1e-5
        # Smoother input constant in k (random across columns): the FP32
        # residual then has no large vertical differences whose rounding the
        # near-singular vertical mode of Dtilde would amplify (eps32 x cond,
        # ~1e-4 here, for fully random u).  b stays random in all directions.
        uh = f32exact(np.broadcast_to(rand(p.og.shape(lev)[1:], 75 + lev), p.og.shape(lev)))
        ud = p.dev(uh, True)
        p.sv.level_smooth(lev, p.dev(b, True), ud, nsweeps=2, rho=0.8, fp32=True)
        assert rel_l2(p.host(ud), p.og.smooth(b, uh, 2, 0.8, lev)) <= 1e-5
        if lev + 1 < p.og.nlevels:
            bc = p.empty(lev + 1, fp32=True)
            p.sv.level_restrict_residual(lev, p.dev(b, True), p.dev(u, True), bc, fp32=True)
            ref = p.og.restrict(p.og.residual(b, u, lev), lev)
            assert rel_l2(p.host(bc), ref) <= 1e-5
            uc = f32exact(rand(p.og.shape(lev + 1), 90 + lev))
            uf = p.dev(u, True)
            p.sv.level_prolong_add(lev, p.dev(uc, True), uf, fp32=True)
            assert rel_l2(p.host(uf), p.og.prolong_add(uc, u, lev)) <= 1e-6


# Levels with n % 32 == 0 (the line smoother's aligned variant: panel-edge
# neighbours written into its staging ring), n % 64 == 0 (the row-staged
# restriction) and n = 48 (the unaligned variant with a separate neighbour
# buffer), on the sphere with both mappings and on the periodic box.
ALIGNED = [
    (1, 64, 16, True, 0, 0.01, 1.0),
    (1, 128, 8, False, 1, 0.05, 4.0),
    (0, 128, 16, True, 0, 0.02, 0.25),
    (1, 48, 16, True, 0, 0.01, 1.0),     # n % 32 != 0 and above the small-level size
]
AIDS = ["sph64", "sph128e", "box128", "sph48"]


@pytest.mark.parametrize("case", ALIGNED, ids=AIDS)
def test_aligned_kernels_fp32(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, precision=1)
    for lev in range(min(2, p.og.nlevels - 1)):
        u = f32exact(rand(p.og.shape(lev), 170 + lev))
        b = f32exact(p.og.volumes(lev) * rand(p.og.shape(lev), 180 + lev))
        bc = p.empty(lev + 1, fp32=True)
        p.sv.level_restrict_residual(lev, p.dev(b, True), p.dev(u, True), bc, fp32=True)
        ref = p.og.restrict(p.og.residual(b, u, lev), lev)
        got = p.host(bc)
        assert rel_l2(got, ref) <= 1e-5, lev
        # element by element as well: a wrong neighbour in one column (a panel
        # corner) hardly moves the L2 norm over thousands of columns
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref)), lev
        uh = f32exact(np.broadcast_to(rand(p.og.shape(lev)[1:], 175 + lev), p.og.shape(lev)))
        ud = p.dev(uh, True)
        p.sv.level_smooth(lev, p.dev(b, True), ud, nsweeps=2, rho=0.8, fp32=True)
        sref = p.og.smooth(b, uh, 2, 0.8, lev)
        sgot = p.host(ud)
        assert rel_l2(sgot, sref) <= 1e-5, lev
        assert np.max(np.abs(sgot - sref)) <= 2e-5 * np.max(np.abs(sref)), lev
        uc = f32exact(rand(p.og.shape(lev + 1), 190 + lev))
        uf = p.dev(u, True)
        p.sv.level_prolong_add(lev, p.dev(uc, True), uf, fp32=True)
        pref = p.og.prolong_add(uc, u, lev)
        pgot = p.host(uf)
        assert rel_l2(pgot, pref) <= 1e-6, lev
        # element by element: panel seams and cube corners
        assert np.max(np.abs(pgot - pref)) <= 1e-6 * np.max(np.abs(pref)), lev


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_vcycles_fp64_fixed_count(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case)
    f = rand(p.og.shape(), 100)
    b = p.og.volumes() * f
    u_ref = p.og.zeros()
    ud = p.empty()
    fd = p.dev(f)
    for _ in range(3):
        p.sv.vcycle(fd, ud)
        u_ref = p.og.vcycle(b, u_ref)
    tol = max(1e-10, fp64_tol(lambda bb: p.og.mg_solve(bb, rtol=0.0, maxit=3)[0], b))
    err = rel_l2(p.host(ud), u_ref)
    print(f"3 V-cycles: err {err:.2e} tol {tol:.2e}")
    assert err <= tol
    # the solve entry point with a fixed count (rtol 0): same iterate
    x = p.empty()
    st, res = p.sv.solve(fd, x, rtol=0.0, maxit=4)
    u4, it, hist = p.og.mg_solve(b, rtol=0.0, maxit=4)
    assert res.iterations == 4 and it == 4
    assert rel_l2(p.host(x), u4) <= tol
    # near the attainable residual two correct FP64 evaluations of b - A x
    # differ by the rounding of the cancelling sum: 16x the oracle's own
    # sensitivity of the residual to ulp-level changes of x
    rfloor = 16.0 * sensitivity(lambda uu: p.og.residual(b, uu), u4) * hist[-1]
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1] + rfloor + 1e-15


@pytest.mark.parametrize("case", CASES[:3], ids=IDS[:3])
def test_pcg_fp64_fixed_count(torch_mod, oracle_mod, case):
    p = make(oracle_mod, case, solver=1)
    f = rand(p.og.shape(), 110)
    b = p.og.volumes() * f
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=0.0, maxit=20)
    u_ref, it, hist = p.og.pcg_solve(b, rtol=0.0, maxit=20)
    assert res.iterations == 20 and it == 20
    tol = max(1e-10, fp64_tol(lambda bb: p.og.pcg_solve(bb, rtol=0.0, maxit=20)[0], b))
    err = rel_l2(p.host(x), u_ref)
    print(f"20 PCG iterations: err {err:.2e} tol {tol:.2e}")
    assert err <= tol
    assert abs(res.rel_residual - hist[-1]) <= 1e-6 * hist[-1]


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_mixed_precision_solution(torch_mod, oracle_mod, case):
    """FP32 V-cycles inside FP64 refinement against the oracle's converged
    FP64 multigrid solution: relative L2 <= 1e-9."""
    p = make(oracle_mod, case, precision=1)
    f = rand(p.og.shape(), 120)
    b = p.og.volumes() * f
    u_ref, it_ref, hist_ref = p.og.mg_solve(b, rtol=1e-13, maxit=80)
    x = p.empty()
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-12, maxit=80)
    err = rel_l2(p.host(x), u_ref)
    print(f"mixed: {res.iterations} cycles, rel residual {res.rel_residual:.2e}, error {err:.2e}")
    assert err <= 1e-9
    assert res.rel_residual <= max(1e-11, 10 * hist_ref[-1])


def test_manufactured_mode_closed_form(torch_mod, oracle_mod):
    """Config-1 box with the Fourier(3,5) x cos(mode 2) right-hand side: the
    mixed solve reproduces the closed-form discrete solution."""
    import sys
    sys.path.insert(0, __file__.rsplit("/", 1)[0])
    from test_oracle_operator import fourier_exact
    n, nz = 32, 32
    p = Pair(oracle_mod, 0, n, nz, precision=1)
    f = inputs.fourier_cos_mode(n, nz)
    x = p.empty()
    # error / residual amplification is ~1e3 here, so iterate to 1e-12
    st, res = p.sv.solve(p.dev(f), x, rtol=1e-12, maxit=50)
    exact = fourier_exact(n, nz, p.r, 0.01, 1.0)
    err = rel_l2(p.host(x), exact)
    print(f"manufactured: {res.iterations} cycles, residual {res.rel_residual:.2e}, error {err:.2e}")
    assert err <= 1e-9


def test_batch_equals_alone(torch_mod, oracle_mod):
    """Members of a batch give bit-identical results to the same solves alone."""
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    # a 32-column-aligned finest level (n = 32) next to unaligned ones, so a
    # batched launch mixes levels the aligned smoother variant would take alone
    specs = [(1, 8, 16, 0.01, 1.0), (0, 24, 12, 0.05, 4.0), (1, 12, 8, 0.002, 0.5),
             (1, 32, 32, 0.01, 1.0), (0, 64, 16, 0.02, 2.0)]
    solvers, rhs = [], []
    for m, (kind, n, nz, w2, l2) in enumerate(specs):
        s = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), w2, l2, precision=1)
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


def test_batch_matches_the_oracle(torch_mod, oracle_mod):
    """Each member of a batched mixed-precision solve (mixed grids, sizes and
    parameters) against the oracle's converged FP64 multigrid solution of its
    own problem: relative L2 <= 1e-9."""
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    specs = [(1, 8, 16, 0.01, 1.0), (0, 24, 12, 0.05, 4.0), (1, 12, 8, 0.002, 0.5),
             (1, 32, 32, 0.01, 1.0), (0, 64, 16, 0.02, 2.0)]
    solvers, rhs, xs = [], [], []
    for m, (kind, n, nz, w2, l2) in enumerate(specs):
        s = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), w2, l2, precision=1)
        solvers.append(s)
        rhs.append(torch.tensor(inputs.uniform_pm1(s.shape(), member=20 + m), device="cuda"))
        xs.append(torch.zeros_like(rhs[-1]))
    st, res = ellsolve.solve_batch(solvers, rhs, xs, rtol=1e-12, maxit=80)
    torch.cuda.synchronize()
    for (kind, n, nz, w2, l2), f, x, r in zip(specs, rhs, xs, res):
        og = oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=True), w2, l2)
        u, _, _ = og.mg_solve(og.volumes() * f.cpu().numpy(), rtol=1e-13, maxit=200)
        err = rel_l2(x.cpu().numpy(), u)
        print(f"batch member {(kind, n, nz)}: {r.iterations} V-cycles, error {err:.2e}")
        assert err <= 1e-9


def test_autotune_changes_no_result(torch_mod, oracle_mod):
    """ellsolve_autotune only changes launch shapes (per level: the smoother's
    occupancy cap, ring depth and tensor-memory use, the transfers' vertical
    split): a solve before and after tuning gives the same bits."""
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    sv = ellsolve.Solver(1, 32, 32, inputs.radial_levels(32, graded=True), 0.01, 1.0, precision=1)
    f = torch.tensor(inputs.uniform_pm1(sv.shape(), member=9), device="cuda")
    x1, x2 = torch.zeros_like(f), torch.zeros_like(f)
    sv.solve(f, x1, rtol=1e-9, maxit=40)
    ctas, ms = sv.autotune()
    assert 2 <= ctas <= 6 and ms > 0
    for level in range(sv.nlevels):
        c, ring, tmem, stg, rc, pc = sv.level_tuning(level)
        print(f"level {level}: ctas {c} ring {ring} tmem {tmem} staged {stg} restrict chunk {rc} "
              f"prolong chunk {pc}")
        assert 0 <= c <= 16 and ring in (4, 8) and tmem in (0, 1, 2) and stg in (0, 1, 2)
        assert rc >= 1 and pc >= 1
    sv.solve(f, x2, rtol=1e-9, maxit=40)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2)


SHAPES = [  # (ctas per SM, ring, tmem, staged, restrict chunk, prolong chunk) on every level
    (3, 8, 0, 0, 608, 608), (5, 4, 2, 2, 152, 152), (4, 8, 1, 2, 1216, 1216),
    (4, 4, 1, 1, 304, 304), (0, 8, 2, 1, 1, 1), (4, 8, 0, 2, 608, 608),
]


@pytest.mark.parametrize("kind,n,nz", [(1, 64, 32), (0, 128, 16), (1, 48, 32)])
def test_every_launch_shape_gives_the_same_bits(torch_mod, oracle_mod, kind, n, nz):
    """Each candidate the autotuner may choose, set on every level, gives a
    solve bit-identical to the default shapes (levels with >= 152 blocks of 128
    columns, the tensor-memory switch forced both ways, the fully staged
    smoother forced both ways, n % 32 == 0 and not)."""
    from paper_1307_2036_gb300 import ellsolve
    torch = torch_mod
    sv = ellsolve.Solver(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.02, 2.0,
                         precision=1)
    f = torch.tensor(inputs.uniform_pm1(sv.shape(), member=19), device="cuda")
    ref = torch.zeros_like(f)
    sv.solve(f, ref, rtol=1e-9, maxit=40)
    for shape in SHAPES:
        for level in range(sv.nlevels):
            sv.set_level_tuning(level, *shape)
        x = torch.zeros_like(f)
        sv.solve(f, x, rtol=1e-9, maxit=40)
        torch.cuda.synchronize()
        assert torch.equal(x, ref), shape
