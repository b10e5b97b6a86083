"""Pins of the oracle's discrete operator (CPU only).

Operator: Eq. ModelEquation integrated over each cell with two-point face
fluxes (Sec. 3.1), Neumann at r = 1 and r = 1 + H; tensor-product form of
Sec. 4.3.1.  Checks that do not reuse the oracle's formula:
  * A 1 = cell volumes (a constant has no flux on any face);
  * symmetry and positive definiteness of the assembled matrix;
  * the assembled matrix and the matrix-free apply agree (two code paths);
  * second-order consistency with the continuous operator on smooth fields;
  * the exact discrete solution for a Fourier mode on the periodic box, from a
    single n_z x n_z solve built here from the shell geometry alone.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs


def make(oracle_mod, kind, n, nz, graded=False, omega2=0.01, lambda2=1.0, mapping=0):
    return oracle_mod.Grid(kind, n, nz, inputs.radial_levels(nz, graded=graded), omega2, lambda2,
                           mapping=mapping)


CASES = [(0, 8, 8, False), (0, 6, 5, True), (1, 4, 6, False), (1, 5, 7, True)]


@pytest.mark.parametrize("kind,n,nz,graded", CASES)
def test_constant_maps_to_volumes(oracle_mod, kind, n, nz, graded):
    g = make(oracle_mod, kind, n, nz, graded, omega2=0.3, lambda2=2.0)
    y = g.apply(np.ones(g.shape()))
    vol = g.volumes()
    assert np.max(np.abs(y - vol) / vol) < 1e-12


@pytest.mark.parametrize("kind,n,nz,graded", CASES)
def test_symmetry(oracle_mod, kind, n, nz, graded):
    g = make(oracle_mod, kind, n, nz, graded, omega2=0.05, lambda2=3.0)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(g.shape()), rng.standard_normal(g.shape())
    xAy, yAx = np.vdot(x, g.apply(y)), np.vdot(y, g.apply(x))
    assert abs(xAy - yAx) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(g.apply(y))


@pytest.mark.parametrize("kind,n,nz,graded", [(0, 4, 8, False), (0, 4, 8, True), (1, 2, 8, True),
                                              (1, 4, 4, False)])
def test_dense_spd_and_matches_apply(oracle_mod, kind, n, nz, graded):
    g = make(oracle_mod, kind, n, nz, graded)
    M = g.dense()
    assert np.max(np.abs(M - M.T)) <= 1e-14 * np.max(np.abs(M))
    np.linalg.cholesky(M)  # raises unless positive definite
    rng = np.random.default_rng(2)
    x = rng.standard_normal(g.shape())
    assert np.allclose(M @ x.reshape(-1), g.apply(x).reshape(-1), rtol=1e-12,
                       atol=1e-14 * np.abs(M).max())
    # off-diagonals are non-positive and rows are strictly diagonally dominant
    off = M - np.diag(np.diag(M))
    assert np.all(off <= 0)
    assert np.all(np.diag(M) > -off.sum(axis=1))


def continuous_box(x, y, r, omega2, lambda2, H):
    """u = cos(3x) cos(2y) cos(pi (r-1)/H) and L u for L of Eq. ModelEquation on the
    flat periodic box (horizontal Laplacian independent of r)."""
    kr = np.pi / H
    w = np.cos(kr * (r - 1))
    dw = -kr * np.sin(kr * (r - 1))
    d2w = -kr * kr * np.cos(kr * (r - 1))
    h = np.cos(3 * x) * np.cos(2 * y)
    u = h * w
    lap_h = -13.0 * u
    radial = h * (d2w + 2.0 * dw / r)
    return u, -omega2 * (lap_h + lambda2 * radial) + u


@pytest.mark.parametrize("omega2,lambda2", [(1.0, 1e-6), (0.01, 1.0)])
def test_second_order_truncation_uniform_box(oracle_mod, omega2, lambda2):
    """(A u)/volume at the cell centres approaches L u at second order on the
    uniform shell."""
    H = 0.01
    errs = []
    for n, nz in [(16, 16), (32, 32), (64, 64)]:
        r = inputs.radial_levels(nz, H=H)
        g = oracle_mod.Grid(0, n, nz, r, omega2, lambda2)
        h = 2 * np.pi / n
        xc = (np.arange(n) + 0.5) * h
        rho = 0.5 * (r[1:] + r[:-1])
        u, Lu = continuous_box(xc[None, None, None, :], xc[None, None, :, None],
                               rho[:, None, None, None], omega2, lambda2, H)
        Au = g.apply(np.broadcast_to(u, g.shape()).copy()) / g.volumes()
        errs.append(np.max(np.abs(Au - Lu)) / np.max(np.abs(Lu)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert errs[-1] < 1e-2
    assert min(rates) > 1.9, (errs, rates)


@pytest.mark.parametrize("omega2,lambda2", [(1.0, 1e-6), (0.01, 1.0)])
def test_second_order_solution_graded_box(oracle_mod, omega2, lambda2):
    """On the graded shell of Eq. VerticalGrading the cell sizes jump by 3x at the
    bottom, so the pointwise truncation error does not vanish; the discrete
    solution for the source L u still converges to u at second order."""
    H = 0.01
    errs = []
    for n, nz in [(8, 16), (16, 32), (32, 64)]:
        r = inputs.radial_levels(nz, H=H, graded=True)
        g = oracle_mod.Grid(0, n, nz, r, omega2, lambda2)
        h = 2 * np.pi / n
        xc = (np.arange(n) + 0.5) * h
        rho = 0.5 * (r[1:] + r[:-1])
        u, Lu = continuous_box(xc[None, None, None, :], xc[None, None, :, None],
                               rho[:, None, None, None], omega2, lambda2, H)
        uh, _, _ = g.mg_solve(g.volumes() * np.broadcast_to(Lu, g.shape()), rtol=1e-12, maxit=80)
        errs.append(np.max(np.abs(uh - u)) / np.max(np.abs(u)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 1.9, (errs, rates)


def fourier_exact(n, nz, r, omega2, lambda2, side=2 * np.pi, kx=3, ky=5, m=2):
    """Exact discrete solution for f = cos(kx x + ky y) cos(pi m (k+1/2)/nz) on the
    periodic box: u = cos(kx x + ky y) v_k, where the horizontal five-point
    difference of the Fourier factor is -mu/h^2 times itself and v solves
    ((h^2 + omega2 mu) V_k) v_k + omega2 lambda2 h^2 [flux terms] = h^2 V_k g_k."""
    h = side / n
    mu = 4 * np.sin(kx * h / 2) ** 2 + 4 * np.sin(ky * h / 2) ** 2
    mid = 0.5 * (r[1:] + r[:-1])
    V = (r[1:] - r[:-1]) / 6.0 * (r[:-1] ** 2 + 4 * mid ** 2 + r[1:] ** 2)  # int r^2 dr
    G = np.zeros(nz + 1)
    G[1:nz] = r[1:nz] ** 2 / (mid[1:] - mid[:-1])
    g = np.cos(np.pi * m * (np.arange(nz) + 0.5) / nz)
    T = np.diag((h * h + omega2 * mu) * V + omega2 * lambda2 * h * h * (G[:-1] + G[1:]))
    T -= np.diag(omega2 * lambda2 * h * h * G[1:nz], 1) + np.diag(omega2 * lambda2 * h * h * G[1:nz], -1)
    v = np.linalg.solve(T, h * h * V * g)
    x = (np.arange(n) + 0.5) * h
    horiz = np.cos(kx * x[None, :] + ky * x[:, None])
    return v[:, None, None, None] * horiz[None, None, :, :]


@pytest.mark.parametrize("n,nz,graded,omega2,lambda2", [(32, 32, False, 0.01, 1.0),
                                                        (16, 24, True, 0.1, 0.01),
                                                        (24, 16, True, 1e-3, 100.0)])
def test_fourier_mode_closed_form(oracle_mod, n, nz, graded, omega2, lambda2):
    r = inputs.radial_levels(nz, graded=graded)
    g = oracle_mod.Grid(0, n, nz, r, omega2, lambda2)
    f = inputs.fourier_cos_mode(n, nz)
    b = g.volumes() * f
    u_exact = fourier_exact(n, nz, r, omega2, lambda2)
    # The operator maps the closed form onto the right-hand side.  The bound is
    # the attainable one: rounding u to FP64 alone leaves ||A (u - fl(u))|| of
    # about eps ||A|| ||u||, here ~1e-11 ||b|| because the vertical coupling
    # exceeds the mass term by ~1e5.
    assert np.linalg.norm(g.apply(u_exact) - b) <= 1e-10 * np.linalg.norm(b)
    # and the multigrid solve reproduces it
    u, it, _ = g.mg_solve(b, rtol=1e-12, maxit=60)
    assert np.linalg.norm(u - u_exact) <= 1e-9 * np.linalg.norm(u_exact)
