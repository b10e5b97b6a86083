"""Pins of the oracle's full multigrid cycle (Sec. 4.3): right-hand side
restricted to every level, the coarsest level smoothed from zero, then on each
finer level the prolongated coarse solution as the start of one V-cycle.

  * it is a linear map of the right-hand side;
  * on a single-level grid it is the coarsest-level sweeps from zero;
  * against the exact discrete solution of a Fourier x vertical mode on the
    box it leaves a smaller algebraic error than one V-cycle from zero, and a
    smaller residual on the seeded uniform right-hand side.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from test_oracle_operator import fourier_exact


def test_fmg_is_linear(oracle_mod):
    g = oracle_mod.Grid(1, 8, 8, inputs.radial_levels(8, graded=True), 0.05, 4.0, coarsest_min=2)
    b1 = g.volumes() * inputs.uniform_pm1(g.shape(), member=21)
    b2 = g.volumes() * inputs.uniform_pm1(g.shape(), member=22)
    lhs = g.fmg(b1 + 2.0 * b2)
    rhs = g.fmg(b1) + 2.0 * g.fmg(b2)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def test_fmg_on_one_level_is_the_coarsest_sweeps(oracle_mod):
    one = oracle_mod.Grid(0, 3, 5, inputs.radial_levels(5), 0.01, 1.0)  # odd n: one level
    assert one.nlevels == 1
    b = one.volumes() * inputs.uniform_pm1(one.shape(), member=23)
    assert np.array_equal(one.fmg(b, nu_coarse=3), one.smooth(b, np.zeros(one.shape()), 3, 1.0))


def test_fmg_beats_one_v_cycle(oracle_mod):
    n, nz = 32, 32
    r = inputs.radial_levels(nz)
    g = oracle_mod.Grid(0, n, nz, r, 0.01, 1.0)
    f = inputs.fourier_cos_mode(n, nz)
    b = g.volumes() * f
    exact = fourier_exact(n, nz, r, 0.01, 1.0)
    e_fmg = np.linalg.norm(g.fmg(b) - exact)
    e_v = np.linalg.norm(g.vcycle(b, np.zeros(g.shape())) - exact)
    assert e_fmg < e_v
    bu = g.volumes() * inputs.uniform_pm1(g.shape(), member=24)
    res = lambda u: np.linalg.norm(g.residual(bu, u)) / np.linalg.norm(bu)  # noqa: E731
    assert res(g.fmg(bu)) < res(g.vcycle(bu, np.zeros(g.shape())))


def test_fmg_two_levels_composes_the_steps(oracle_mod):
    """Two levels: restrict b, coarse sweeps from zero, interpolate onto a zero
    fine field, one V-cycle from there (Sec. 4.3)."""
    for n in (8, 12):
        g = oracle_mod.Grid(0, n, 6, inputs.radial_levels(6, graded=True), 0.02, 2.0)
        if g.nlevels == 2:
            break
    assert g.nlevels == 2
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=25)
    for mode in (0, 1):
        bc = g.restrict(b)
        uc = g.smooth(bc, np.zeros(g.shape(1)), 3, 1.0, lev=1)
        u0 = g.prolong_add(uc, np.zeros(g.shape()), 0, mode=mode)
        want = g.vcycle(b, u0, nu_coarse=3, prolong_mode=mode)
        got = g.fmg(b, nu_coarse=3, prolong_mode=mode)
        assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


def test_mg_solve_first_cycle_is_fmg(oracle_mod):
    """With the flag set, multigrid's first cycle is the full multigrid cycle and
    the later ones V-cycles from its result."""
    r = inputs.radial_levels(8, graded=True)
    g = oracle_mod.Grid(1, 8, 8, r, 0.05, 4.0, fmg=True)
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=26)
    u1 = g.mg_solve(b, rtol=0.0, maxit=1)[0]
    assert np.array_equal(u1, g.fmg(b))
    u3 = g.mg_solve(b, rtol=0.0, maxit=3)[0]
    assert np.array_equal(u3, g.vcycle(b, g.vcycle(b, u1)))
    # and it converges to the same solution as plain multigrid
    plain = oracle_mod.Grid(1, 8, 8, r, 0.05, 4.0)
    ua, ita, _ = g.mg_solve(b, rtol=1e-12, maxit=60)
    ub, itb, _ = plain.mg_solve(b, rtol=1e-12, maxit=60)
    assert np.linalg.norm(ua - ub) <= 1e-10 * np.linalg.norm(ub)
    assert ita <= itb


@pytest.mark.parametrize("kind,n", [(0, 8), (1, 8)])
def test_fmg_preconditioned_cg_equals_dense_lu(oracle_mod, kind, n):
    g = oracle_mod.Grid(kind, n, 4, inputs.radial_levels(4, graded=True), 0.05, 4.0, precond=2,
                        mg_precond=(2, 2, 2, 0.8, 0), fmg=True)
    b = g.volumes() * inputs.uniform_pm1(g.shape(), member=27)
    u, it, hist = g.pcg_solve(b, rtol=1e-13, maxit=50)
    exact = np.linalg.solve(g.dense(), b.reshape(-1))
    assert np.linalg.norm(u.reshape(-1) - exact) <= 1e-10 * np.linalg.norm(exact)
