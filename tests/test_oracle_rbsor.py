"""Pins of the oracle's block red-black SOR smoother and block red-black SSOR
preconditioner (Sec. 4.2, Eq. BlockRBSOR; Sec. 6.2.1 colouring; Sec. 7.2 CG
preconditioner), each against a formula the oracle does not compute:

  * on the periodic box one sweep is block Gauss-Seidel in red-black order,
    with relaxation, on the dense matrix: x_R <- (1-rho) x_R + rho A_RR^{-1}
    (b_R - A_RB x_B), then the same for the black unknowns;
  * on the cubed sphere (no two-colouring exists: three cells meet pairwise
    at a cube corner) a sweep is x <- x + rho P_R D^{-1} (b - A x), then the
    same with P_B, D the column-block diagonal of the dense matrix;
  * the SSOR preconditioner, assembled column by column, is symmetric and
    positive definite;
  * the converged multigrid solution with this smoother equals dense LU;
  * the paper's observations: the multigrid needs fewer V-cycles with block
    RB-SOR than with block Jacobi (Table 7 against Table 3), and CG fewer
    iterations with RB-SSOR than with block Jacobi.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs


def grid(oracle_mod, kind, n, nz, graded=False, w2=0.05, l2=4.0, **kw):
    return oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=graded), w2, l2,
                           coarsest_min=kw.pop("coarsest_min", 4), **kw)


def unknown_colour(g):
    return np.tile(g.colour(), g.nz)  # layout k * ncol + c


def column_block_diagonal(g, A):
    """Keep only the couplings inside a vertical column."""
    col = np.tile(np.arange(g.ncol()), g.nz)
    return np.where(col[:, None] == col[None, :], A, 0.0)


@pytest.mark.parametrize("n,nz,graded,rho", [(4, 4, False, 1.0), (6, 3, True, 1.3),
                                             (4, 5, True, 0.7)])
def test_box_sweep_is_red_black_block_gauss_seidel(oracle_mod, n, nz, graded, rho):
    g = grid(oracle_mod, 0, n, nz, graded, smoother=1)
    A = g.dense()
    b = g.volumes().reshape(-1) * inputs.uniform_pm1(g.shape(), member=1).reshape(-1)
    x = inputs.uniform_pm1(g.shape(), member=2).reshape(-1)
    col = unknown_colour(g)
    R, B = np.where(col == 0)[0], np.where(col == 1)[0]
    # no red column couples to another red column on the box
    assert np.all(column_block_diagonal(g, A)[np.ix_(R, R)] == A[np.ix_(R, R)])
    y = x.copy()
    y[R] = (1 - rho) * y[R] + rho * np.linalg.solve(A[np.ix_(R, R)], b[R] - A[np.ix_(R, B)] @ y[B])
    y[B] = (1 - rho) * y[B] + rho * np.linalg.solve(A[np.ix_(B, B)], b[B] - A[np.ix_(B, R)] @ y[R])
    got = g.smooth(b, x, nsweeps=1, rho=rho).reshape(-1)
    assert np.max(np.abs(got - y)) <= 1e-10 * np.max(np.abs(y))


@pytest.mark.parametrize("n,mapping", [(2, 0), (4, 1)])
def test_sphere_sweep_updates_each_colour_from_the_current_iterate(oracle_mod, n, mapping):
    g = grid(oracle_mod, 1, n, 3, True, mapping=mapping, smoother=1, coarsest_min=1)
    A = g.dense()
    D = column_block_diagonal(g, A)
    b = g.volumes().reshape(-1) * inputs.uniform_pm1(g.shape(), member=3).reshape(-1)
    x = inputs.uniform_pm1(g.shape(), member=4).reshape(-1)
    col = unknown_colour(g)
    rho = 1.1
    y = x.copy()
    for colour in (0, 1):
        e = np.linalg.solve(D, b - A @ y)
        y = y + rho * np.where(col == colour, e, 0.0)
    got = g.smooth(b, x, nsweeps=1, rho=rho).reshape(-1)
    assert np.max(np.abs(got - y)) <= 1e-10 * np.max(np.abs(y))
    # on the sphere some same-colour columns are neighbours (it is not a
    # two-colouring), which is why the half-sweep is defined this way
    same = (A != 0) & (D == 0) & (col[:, None] == col[None, :])
    assert same.any()


@pytest.mark.parametrize("kind,n", [(0, 4), (1, 2)])
def test_rb_ssor_preconditioner_is_symmetric_positive_definite(oracle_mod, kind, n):
    g = grid(oracle_mod, kind, n, 4, True, coarsest_min=1)
    N = g.ncol() * g.nz
    M = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = g.rb_ssor(e.reshape(g.shape()), rho=1.0).reshape(-1)
    assert np.max(np.abs(M - M.T)) <= 1e-12 * np.max(np.abs(M))
    assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0


@pytest.mark.parametrize("kind,n", [(0, 8), (1, 8)])
def test_rb_multigrid_solution_equals_dense_lu(oracle_mod, kind, n):
    g = grid(oracle_mod, kind, n, 4, True, smoother=1)
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=5)
    u, it, hist = g.mg_solve(b, rtol=1e-13, maxit=60, nu_pre=1, nu_post=1, rho=1.0)
    exact = np.linalg.solve(g.dense(), b.reshape(-1))
    assert np.linalg.norm(u.reshape(-1) - exact) <= 1e-10 * np.linalg.norm(exact)


def test_rb_sor_needs_fewer_v_cycles_than_jacobi(oracle_mod):
    r = inputs.radial_levels(32)
    f = inputs.uniform_pm1((32, 1, 32, 32), member=6)
    its = {}
    for smoother, rho in ((0, 0.8), (1, 1.0)):
        g = oracle_mod.Grid(0, 32, 32, r, 0.01, 1.0, smoother=smoother)
        _, it, _ = g.mg_solve(g.volumes() * f, rtol=1e-5, maxit=50, nu_pre=1, nu_post=1, rho=rho)
        its[smoother] = it
    assert its[1] < its[0], its


def test_pcg_with_rb_ssor_needs_fewer_iterations(oracle_mod):
    r = inputs.radial_levels(16, graded=True)
    f = inputs.uniform_pm1((16, 1, 32, 32), member=7)
    its = {}
    for pc in (0, 1):
        g = oracle_mod.Grid(0, 32, 16, r, 0.05, 1.0, precond=pc)
        _, it, hist = g.pcg_solve(g.volumes() * f, rtol=1e-8, maxit=500)
        assert hist[-1] < 1e-8
        its[pc] = it
    assert its[1] < its[0], its
