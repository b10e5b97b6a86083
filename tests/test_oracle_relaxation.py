"""Pins of the oracle's tridiagonal solves, line relaxation and intergrid
transfers (CPU only).

  * Algorithm Thomas (both groupings of its denominator) against dense LU, and
    against a 60-digit solve (mpmath) on the stiffest column of the graded
    shell, where the printed grouping loses digits and the excess grouping
    must not;
  * one line-relaxation sweep equals u + rho * Dtilde^{-1}(b - A u), with
    Dtilde cut out of the assembled matrix as its vertical tridiagonal blocks
    (Sec. 4.2) and solved densely;
  * restriction conserves the integrated residual; prolongation reproduces
    constants everywhere (cube corners included) and linear fields inside a
    panel (Sec. 6.2.1: cell average / linear interpolation).
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs


def random_mmatrix(n, rng, excess_scale=1.0):
    up = rng.uniform(0.5, 2.0, n)
    lo = rng.uniform(0.5, 2.0, n)
    up[-1] = 0.0
    lo[0] = 0.0
    delta = excess_scale * rng.uniform(0.1, 1.0, n)
    M = np.diag(delta + up + lo) - np.diag(up[:-1], 1) - np.diag(lo[1:], -1)
    return delta, up, lo, M


@pytest.mark.parametrize("n", [1, 2, 3, 17, 128])
def test_thomas_against_dense(oracle_mod, n):
    rng = np.random.default_rng(n)
    delta, up, lo, M = random_mmatrix(n, rng)
    f = rng.standard_normal(n)
    ref = np.linalg.solve(M, f)
    a, b, c = np.diag(M).copy(), np.zeros(n), np.zeros(n)
    b[:-1] = -up[:-1]
    c[1:] = -lo[1:]
    assert np.allclose(oracle_mod.thomas_paper(a, b, c, f), ref, rtol=1e-12, atol=1e-13)
    assert np.allclose(oracle_mod.thomas_excess(delta, up, lo, f), ref, rtol=1e-12, atol=1e-13)


def test_thomas_diagonal_exact(oracle_mod):
    n = 9
    d = np.arange(1.0, n + 1)
    f = d * np.linspace(-2, 3, n)
    z = np.zeros(n)
    assert np.array_equal(oracle_mod.thomas_excess(d, z, z, f), f / d)
    assert np.array_equal(oracle_mod.thomas_paper(d, z, z, f), f / d)


def test_thomas_excess_accurate_on_graded_shell(oracle_mod):
    mp = pytest.importorskip("mpmath")
    nz = 128
    r = inputs.radial_levels(nz, graded=True)
    g = oracle_mod.Grid(1, 8, nz, r, 0.01, 1.0)
    V, G = g.radial()
    area, trans, _ = g.geometry()
    A, sT = area[0], trans[0].sum()
    wl2 = 0.01
    delta = A * V + 0.01 * V * sT
    up = wl2 * A * G[1:]
    lo = wl2 * A * G[:-1]
    f = np.random.default_rng(5).standard_normal(nz) * A * V
    mp.mp.dps = 60
    Mm = mp.matrix(nz, nz)
    for k in range(nz):
        Mm[k, k] = mp.mpf(delta[k]) + mp.mpf(up[k]) + mp.mpf(lo[k])
        if k + 1 < nz:
            Mm[k, k + 1] = -mp.mpf(up[k])
            Mm[k + 1, k] = -mp.mpf(lo[k + 1])
    exact = np.array([float(v) for v in mp.lu_solve(Mm, mp.matrix([mp.mpf(x) for x in f]))])
    err_excess = np.linalg.norm(oracle_mod.thomas_excess(delta, up, lo, f) - exact) / np.linalg.norm(exact)
    a = delta + up + lo
    b = -np.append(up[:-1], 0.0)
    c = -np.insert(lo[1:], 0, 0.0)
    err_paper = np.linalg.norm(oracle_mod.thomas_paper(a, b, c, f) - exact) / np.linalg.norm(exact)
    assert err_excess < 1e-13, err_excess
    assert err_paper > 10 * err_excess  # the reason for the excess grouping


def tridiagonal_blocks(M, ncol, nz):
    """Dtilde: keep the entries of M that couple cells of the same column."""
    D = np.zeros_like(M)
    for c in range(ncol):
        idx = [k * ncol + c for k in range(nz)]
        D[np.ix_(idx, idx)] = M[np.ix_(idx, idx)]
    return D


@pytest.mark.parametrize("kind,n,nz,graded", [(0, 4, 8, False), (1, 2, 6, True)])
def test_line_jacobi_sweep_is_block_jacobi(oracle_mod, kind, n, nz, graded):
    g = oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=graded), 0.05, 2.0)
    M = g.dense()
    D = tridiagonal_blocks(M, g.ncol(), nz)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(g.shape()) * g.volumes()
    u0 = rng.standard_normal(g.shape())
    # Backward error: rho^{-1} Dtilde (u1 - u0) reproduces b - A u0 to rounding;
    # forward error within eps * cond(Dtilde) of the dense solve.
    rhs = b.reshape(-1) - M @ u0.reshape(-1)
    bound = 64 * np.finfo(float).eps * np.linalg.cond(D)
    for rho in (1.0, 0.8):
        step = (g.smooth(b, u0, nsweeps=1, rho=rho) - u0).reshape(-1) / rho
        assert np.linalg.norm(D @ step - rhs) <= 1e-14 * np.linalg.norm(np.abs(D) @ np.abs(step))
        ref = np.linalg.solve(D, rhs)
        assert np.linalg.norm(step - ref) <= bound * np.linalg.norm(ref)
    z = g.line_precond(b).reshape(-1)
    assert np.linalg.norm(D @ z - b.reshape(-1)) <= 1e-14 * np.linalg.norm(np.abs(D) @ np.abs(z))
    u2 = g.smooth(b, u0, nsweeps=2, rho=0.8)
    assert np.allclose(u2, g.smooth(b, g.smooth(b, u0, 1, 0.8), 1, 0.8), rtol=1e-14, atol=0)


@pytest.mark.parametrize("kind,n", [(0, 8), (1, 8)])
def test_restriction_conserves_integral(oracle_mod, kind, n):
    g = oracle_mod.Grid(kind, n, 3, inputs.radial_levels(3), 0.01, 1.0)
    r = np.random.default_rng(4).standard_normal(g.shape(0))
    bc = g.restrict(r, 0)
    assert np.allclose(bc.sum(axis=(1, 2, 3)), r.sum(axis=(1, 2, 3)), rtol=1e-13, atol=1e-13)
    # a single fine value lands on its parent only
    d = np.zeros(g.shape(0))
    d[1, -1, 5, 2] = 2.5
    e = g.restrict(d, 0)
    assert e[1, -1, 2, 1] == 2.5 and np.count_nonzero(e) == 1


@pytest.mark.parametrize("kind,n", [(0, 8), (1, 8), (1, 4)])
def test_prolongation_reproduces_constants(oracle_mod, kind, n):
    g = oracle_mod.Grid(kind, n, 2, inputs.radial_levels(2), 0.01, 1.0, coarsest_min=2)
    for mode in (0, 1):
        uf = g.prolong_add(np.full(g.shape(1), 3.0), np.zeros(g.shape(0)), 0, mode=mode)
        assert np.allclose(uf, 3.0, rtol=1e-15)


def test_prolongation_linear_and_weights_on_box(oracle_mod):
    n = 16
    g = oracle_mod.Grid(0, n, 1, inputs.radial_levels(1), 0.01, 1.0)
    nc = n // 2
    I, J = np.meshgrid(np.arange(nc), np.arange(nc))
    # coarse centre of (I, J) sits at fine index coordinate 2I + 1/2
    uc = (0.3 * (2 * I + 0.5) - 1.7 * (2 * J + 0.5) + 4.0)[None, None]
    uf = g.prolong_add(uc, np.zeros(g.shape(0)), 0)
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    lin = 0.3 * i - 1.7 * j + 4.0
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(uf[0, 0][inner], lin[inner], rtol=1e-14)
    # a coarse delta spreads with the bilinear weights 9, 3, 3, 1 (/16)
    d = np.zeros(g.shape(1))
    d[0, 0, 3, 3] = 16.0
    e = g.prolong_add(d, np.zeros(g.shape(0)), 0)[0, 0]
    block = e[5:9, 5:9]
    expect = np.array([[1, 3, 3, 1], [3, 9, 9, 3], [3, 9, 9, 3], [1, 3, 3, 1]], float)
    assert np.array_equal(block, expect)
    assert e.sum() == 64.0


def test_prolongation_cube_corner_weights(oracle_mod):
    """At a cube corner only three coarse cells meet; the corner child gets
    1/2 of its parent and 1/4 of each of the two neighbours across the edges."""
    g = oracle_mod.Grid(1, 4, 1, inputs.radial_levels(1), 0.01, 1.0, coarsest_min=2)
    nc = 2
    _, _, nbr_c = g.geometry(1)
    parent = 0  # panel 0, (I, J) = (0, 0); fine child (0, 0) points to -i and -j
    X, Y = nbr_c[parent, 0], nbr_c[parent, 2]
    uc = np.zeros(g.shape(1))
    uc.reshape(-1)[parent] = 8.0
    uc.reshape(-1)[X] = 4.0
    uc.reshape(-1)[Y] = 2.0
    uf = g.prolong_add(uc, np.zeros(g.shape(0)), 0)
    assert uf.reshape(-1)[0] == 0.5 * 8 + 0.25 * 4 + 0.25 * 2
    assert nc * nc * 6 == g.ncol(1)
