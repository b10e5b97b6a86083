"""Pins of the oracle's CG preconditioned by one multigrid V-cycle (Sec. 4.3:
multigrid as a preconditioner for a Krylov method), with the flexible
(Polak-Ribiere) beta:

  * it converges to the dense LU solution;
  * it needs no more iterations than the multigrid alone, and far fewer than
    CG with block Jacobi;
  * why beta is the flexible one: the V-cycle as an operator M^{-1} is
    symmetric with piecewise-constant prolongation (then the 2x2 sum is its
    transpose) and damped block Jacobi, and not symmetric with the bilinear
    prolongation.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs


def grid(oracle_mod, kind, n, nz, prolong=0, **kw):
    return oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.05, 4.0,
                           precond=2, mg_precond=(2, 2, 2, 0.8, prolong), **kw)


@pytest.mark.parametrize("kind,n", [(0, 8), (1, 8)])
def test_mg_pcg_equals_dense_lu(oracle_mod, kind, n):
    g = grid(oracle_mod, kind, n, 4)
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=11)
    u, it, hist = g.pcg_solve(b, rtol=1e-13, maxit=50)
    exact = np.linalg.solve(g.dense(), b.reshape(-1))
    assert np.linalg.norm(u.reshape(-1) - exact) <= 1e-10 * np.linalg.norm(exact)


@pytest.mark.parametrize("kind,n,nz", [(0, 32, 32), (1, 16, 16)])
def test_mg_pcg_iterations(oracle_mod, kind, n, nz):
    g = grid(oracle_mod, kind, n, nz)
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=12)
    _, it_cg, h = g.pcg_solve(b, rtol=1e-8, maxit=100)
    assert h[-1] < 1e-8
    _, it_mg, _ = g.mg_solve(b, rtol=1e-8, maxit=100)
    j = oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=True), 0.05, 4.0)
    _, it_jac, _ = j.pcg_solve(b, rtol=1e-8, maxit=1000)
    assert it_cg <= it_mg, (it_cg, it_mg)
    assert 3 * it_cg < it_jac, (it_cg, it_jac)


@pytest.mark.parametrize("prolong,symmetric", [(1, True), (0, False)])
def test_v_cycle_operator_symmetry(oracle_mod, prolong, symmetric):
    g = oracle_mod.Grid(0, 8, 3, inputs.radial_levels(3), 0.05, 4.0)
    N = g.ncol() * g.nz
    M = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        M[:, j] = g.vcycle(e.reshape(g.shape()), np.zeros(g.shape()), 2, 2, 2, 0.8, 1.0,
                           prolong).reshape(-1)
    asym = np.max(np.abs(M - M.T)) / np.max(np.abs(M))
    if symmetric:
        assert asym <= 1e-12
        assert np.min(np.linalg.eigvalsh(0.5 * (M + M.T))) > 0
    else:
        assert asym > 1e-6
