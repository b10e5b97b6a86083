"""Pins of the oracle's vertical background profiles (Sec. 2, the operator
D^(z) of Eq. FullSISLEquation; the equation multiplied by p(r) r^2 so that the
discrete operator stays symmetric): V_k -> V_k p_cell[k], G_k -> G_k q_face[k].

  * unit profiles give the model equation bit for bit;
  * the operator is symmetric positive definite, and its row sums are the
    weighted volumes A_P V_k p_k (the Laplacian parts annihilate constants);
  * a Fourier x vertical mode on the periodic box is solved exactly by an
    independent n_z x n_z solve built from the weighted coefficients;
  * the multigrid keeps its iteration count (the paper expects its solvers to
    be robust to this generalisation).
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from test_oracle_operator import fourier_exact  # noqa: F401  (same closed form, unit profiles)


def profiles(nz, r):
    """Smooth positive profiles of the radius: p from a decaying background,
    q = p / (1 + c N^2(r)) at the interfaces."""
    mid = 0.5 * (r[1:] + r[:-1])
    s = (mid - r[0]) / (r[-1] - r[0])
    p_cell = np.exp(-1.5 * s) * (1.0 + 0.2 * np.sin(3 * np.pi * s))
    t = (r - r[0]) / (r[-1] - r[0])
    q_face = np.exp(-1.5 * t) / (1.0 + 0.8 * (1.0 + np.cos(2 * np.pi * t)))
    return p_cell, q_face


def fourier_exact_profiles(n, nz, r, omega2, lambda2, p_cell, q_face, kx=3, ky=5, m=2):
    """As fourier_exact, with V_k and G_k weighted by the profiles."""
    h = 2 * np.pi / n
    mu = 4 * np.sin(kx * h / 2) ** 2 + 4 * np.sin(ky * h / 2) ** 2
    mid = 0.5 * (r[1:] + r[:-1])
    V = (r[1:] - r[:-1]) / 6.0 * (r[:-1] ** 2 + 4 * mid ** 2 + r[1:] ** 2) * p_cell
    G = np.zeros(nz + 1)
    G[1:nz] = r[1:nz] ** 2 / (mid[1:] - mid[:-1]) * q_face[1:nz]
    g = np.cos(np.pi * m * (np.arange(nz) + 0.5) / nz)
    T = np.diag((h * h + omega2 * mu) * V + omega2 * lambda2 * h * h * (G[:-1] + G[1:]))
    T -= np.diag(omega2 * lambda2 * h * h * G[1:nz], 1) + np.diag(omega2 * lambda2 * h * h * G[1:nz], -1)
    v = np.linalg.solve(T, h * h * V * g)
    x = (np.arange(n) + 0.5) * h
    horiz = np.cos(kx * x[None, :] + ky * x[:, None])
    return v[:, None, None, None] * horiz[None, None, :, :]


def test_unit_profiles_are_the_model_equation(oracle_mod):
    nz = 8
    r = inputs.radial_levels(nz, graded=True)
    a = oracle_mod.Grid(1, 8, nz, r, 0.01, 1.0)
    b = oracle_mod.Grid(1, 8, nz, r, 0.01, 1.0, p_cell=np.ones(nz), q_face=np.ones(nz + 1))
    u = inputs.uniform_pm1(a.shape(), member=1)
    assert np.array_equal(a.apply(u), b.apply(u))
    assert np.array_equal(a.volumes(), b.volumes())


@pytest.mark.parametrize("kind,n,nz", [(0, 4, 6), (1, 2, 4)])
def test_profiles_operator_spd_and_row_sums(oracle_mod, kind, n, nz):
    r = inputs.radial_levels(nz, graded=True)
    pc, qf = profiles(nz, r)
    g = oracle_mod.Grid(kind, n, nz, r, 0.05, 4.0, coarsest_min=1, p_cell=pc, q_face=qf)
    A = g.dense()
    assert np.max(np.abs(A - A.T)) <= 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)
    plain = oracle_mod.Grid(kind, n, nz, r, 0.05, 4.0, coarsest_min=1)
    expect = (plain.volumes() * pc[:, None, None, None]).reshape(-1)
    # the row sums cancel against a diagonal ~1e5 times larger: bound the
    # rounding by the absolute row sums
    assert np.max(np.abs(A.sum(axis=1) - expect) / np.abs(A).sum(axis=1)) <= 1e-14


@pytest.mark.parametrize("n,nz,graded,omega2,lambda2", [(32, 32, False, 0.01, 1.0),
                                                        (16, 24, True, 0.1, 0.01)])
def test_profiles_fourier_mode_closed_form(oracle_mod, n, nz, graded, omega2, lambda2):
    r = inputs.radial_levels(nz, graded=graded)
    pc, qf = profiles(nz, r)
    g = oracle_mod.Grid(0, n, nz, r, omega2, lambda2, p_cell=pc, q_face=qf)
    f = inputs.fourier_cos_mode(n, nz)
    b = g.volumes() * f
    u_exact = fourier_exact_profiles(n, nz, r, omega2, lambda2, pc, qf)
    assert np.linalg.norm(g.apply(u_exact) - b) <= 1e-10 * np.linalg.norm(b)
    u, it, _ = g.mg_solve(b, rtol=1e-12, maxit=60)
    assert np.linalg.norm(u - u_exact) <= 1e-9 * np.linalg.norm(u_exact)


def test_multigrid_robust_to_profiles(oracle_mod):
    nz = 32
    r = inputs.radial_levels(nz, graded=True)
    pc, qf = profiles(nz, r)
    f = inputs.uniform_pm1((nz, 6, 16, 16), member=3)
    its = []
    for kw in ({}, {"p_cell": pc, "q_face": qf}):
        g = oracle_mod.Grid(1, 16, nz, r, 0.01, 1.0, **kw)
        _, it, _ = g.mg_solve(g.volumes() * f, rtol=1e-8, maxit=50)
        its.append(it)
    assert its[1] <= its[0] + 2, its
