"""Pins of the oracle's sphere metric: cell centres, centre distances d_PQ, face
lengths l_PQ and the transmissibilities T_PQ = l_PQ / d_PQ (CPU only).

The reading (Sec. 3.1, Eqs. x1x2_1 / x1x2_2): a cell's centre is the image of
the mid-point of its coordinate rectangle under the panel's mapping, and l and
d are great-circle arcs on the unit sphere.  The checks below use facts the
oracle's code does not compute:
  * the centre's mapping coordinates, recovered from the oracle's centre by
    the inverse mapping (atan2 of the panel components), are the mid-points
    (i + 1/2), (j + 1/2) of the coordinate grid;
  * points rebuilt from the angular form cos(a)cos(b) N + sin(a)cos(b) A +
    cos(a)sin(b) B (no tangent, unlike the oracle), and their arcs by
    atan2(|a x b|, a . b) (the oracle uses the chord and asin), give l, d and
    T to rounding, on every level of the hierarchy (coarse centres are
    recomputed on the coarse grid, not averaged);
  * the discrete operator's horizontal part is consistent with the
    Laplace-Beltrami operator where the grid is orthogonal (the panel-centre
    cell of an odd grid): for spherical harmonics Y of degree l,
    Delta_S Y = -l(l+1) Y, and the truncation error there falls at second
    order;
  * on the whole sphere the solution error of -omega^2 Delta_S u + u = f for a
    spherical harmonic stays a few percent and does not shrink as n doubles
    (observed order 0): the two-point fluxes of the 7-point stencil are not
    consistent on the skewed cells along the panel edges (Sec. 3.1 notes the
    grid is non-orthogonal), so this test bounds the error instead of
    asserting an order.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs

# Panel frames (normal N, axes A, B with A x B = N): the numbering convention of
# the cell index c = (p n + j) n + i (a data-layout definition).
N_ = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
A_ = np.array([[0, 1, 0], [-1, 0, 0], [0, -1, 0], [1, 0, 0], [0, 1, 0], [0, 1, 0]], float)
B_ = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1], [-1, 0, 0], [1, 0, 0]], float)


def grid(oracle_mod, n, mapping, nz=1, omega2=1.0, coarsest_min=1):
    return oracle_mod.Grid(1, n, nz, inputs.radial_levels(nz), omega2, 1.0, mapping=mapping,
                           coarsest_min=coarsest_min)


def angle_of_line(t, n, mapping):
    """Angle a with tan(a) = mapping coordinate of grid line t (t may be half-integer)."""
    t = np.asarray(t, float)
    if mapping == 1:
        return np.arctan(-1.0 + 2.0 * t / n)
    return -np.pi / 4 + t * (np.pi / 2) / n


def point(p, a, b):
    """Unit vector with panel angles (a, b): the direction of N + tan(a) A + tan(b) B,
    written without tangents."""
    a = np.asarray(a, float)[..., None]
    b = np.asarray(b, float)[..., None]
    X = np.cos(a) * np.cos(b) * N_[p] + np.sin(a) * np.cos(b) * A_[p] + np.cos(a) * np.sin(b) * B_[p]
    return X / np.linalg.norm(X, axis=-1, keepdims=True)


def arc(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def ref_centres(n, mapping):
    """(6 n n, 3) centres rebuilt from the mid-point angles."""
    out = np.empty((6, n, n, 3))
    mid = angle_of_line(np.arange(n) + 0.5, n, mapping)
    for p in range(6):
        out[p] = point(p, mid[None, :], mid[:, None])  # [j, i]
    return out.reshape(-1, 3)


def ref_corners(n, mapping):
    """(6 n n, 4, 3) corners (i, j), (i+1, j), (i, j+1), (i+1, j+1)."""
    t = angle_of_line(np.arange(n + 1), n, mapping)
    out = np.empty((6, n, n, 4, 3))
    for p in range(6):
        X = point(p, t[None, :], t[:, None])  # [j, i]
        out[p, :, :, 0] = X[:-1, :-1]
        out[p, :, :, 1] = X[:-1, 1:]
        out[p, :, :, 2] = X[1:, :-1]
        out[p, :, :, 3] = X[1:, 1:]
    return out.reshape(-1, 4, 3)


@pytest.mark.parametrize("mapping", [0, 1])
@pytest.mark.parametrize("n", [1, 3, 8, 12])
def test_centres_are_mapped_midpoints(oracle_mod, n, mapping):
    g = grid(oracle_mod, n, mapping)
    for lev in range(g.nlevels):
        m = g.level_n(lev)
        X = g.centres(lev).reshape(6, m, m, 3)
        assert np.abs(np.linalg.norm(X, axis=-1) - 1).max() < 1e-15
        mid = angle_of_line(np.arange(m) + 0.5, m, mapping)
        for p in range(6):
            xn, xa, xb = X[p] @ N_[p], X[p] @ A_[p], X[p] @ B_[p]
            assert xn.min() > 0
            # inverse mapping: the angles whose tangents are the coordinates
            assert np.abs(np.arctan2(xa, xn) - mid[None, :]).max() < 1e-14, (lev, p)
            assert np.abs(np.arctan2(xb, xn) - mid[:, None]).max() < 1e-14, (lev, p)


@pytest.mark.parametrize("mapping", [0, 1])
def test_centre_is_not_the_corner_average(oracle_mod, mapping):
    """Sensitivity of the centre pin: the normalised average of the corners (a
    plausible mistake) differs from the mapped mid-point by far more than the
    tolerance used above."""
    n = 8
    X = grid(oracle_mod, n, mapping).centres()
    avg = ref_corners(n, mapping).mean(axis=1)
    avg /= np.linalg.norm(avg, axis=-1, keepdims=True)
    assert np.abs(avg - X).max() > 1e-5


@pytest.mark.parametrize("mapping", [0, 1])
@pytest.mark.parametrize("n", [2, 4, 16])
def test_distances_lengths_and_transmissibilities(oracle_mod, n, mapping):
    g = grid(oracle_mod, n, mapping)
    # faces -i, +i, -j, +j as corner pairs
    pairs = [(0, 2), (1, 3), (0, 1), (2, 3)]
    for lev in range(g.nlevels):
        m = g.level_n(lev)
        _, trans, nbr = g.geometry(lev)
        ell, dist = g.face_lengths(lev)
        C = ref_centres(m, mapping)
        K = ref_corners(m, mapping)
        for q, (a, b) in enumerate(pairs):
            l_ref = arc(K[:, a], K[:, b])
            d_ref = arc(C, C[nbr[:, q]])
            assert np.abs(ell[:, q] - l_ref).max() < 1e-14, (lev, q)
            assert np.abs(dist[:, q] - d_ref).max() < 1e-14, (lev, q)
            assert np.abs(trans[:, q] / (l_ref / d_ref) - 1).max() < 1e-12, (lev, q)


def test_arc_is_not_the_chord(oracle_mod):
    """Sensitivity of the distance pin: the chord between the centres (a
    plausible mistake) differs from the arc by far more than 1e-14."""
    n = 4
    g = grid(oracle_mod, n, 0)
    _, _, nbr = g.geometry()
    C = ref_centres(n, 0)
    chord = np.linalg.norm(C - C[nbr[:, 0]], axis=-1)
    assert np.abs(chord - arc(C, C[nbr[:, 0]])).min() > 1e-3


def _harmonics():
    # homogeneous harmonic polynomials restricted to the unit sphere, degree l
    return [
        (1, lambda X: X[..., 2] + 0.5 * X[..., 0]),
        (2, lambda X: X[..., 0] ** 2 - X[..., 1] ** 2 + X[..., 1] * X[..., 2]),
        (3, lambda X: X[..., 0] * X[..., 1] * X[..., 2] + X[..., 0] * (5 * X[..., 2] ** 2 - 1)),
    ]


@pytest.mark.parametrize("mapping", [0, 1])
@pytest.mark.parametrize("l,Y", _harmonics())
def test_laplace_beltrami_second_order_at_panel_centres(oracle_mod, mapping, l, Y):
    """One level, nz = 1: (A u)/(A_P V_0) = u - omega^2 Delta_h u.  At the
    panel-centre cell of an odd grid (orthogonal and symmetric there)
    -Delta_h Y approaches l(l+1) Y at second order in 1/n."""
    errs, ns = [], [9, 19, 39, 79]
    for n in ns:
        g = grid(oracle_mod, n, mapping)
        y = Y(g.centres())
        lap = (g.apply(y.reshape(1, 6, n, n)) / g.volumes()).reshape(6, n, n) - y.reshape(6, n, n)
        c = (n - 1) // 2
        errs.append(np.abs(lap[:, c, c] - l * (l + 1) * y.reshape(6, n, n)[:, c, c]).max())
    rates = [np.log(errs[i] / errs[i + 1]) / np.log(ns[i + 1] / ns[i]) for i in range(3)]
    print(f"mapping {mapping} degree {l}: truncation at panel centres {errs}, orders {rates}")
    assert min(rates) > 1.9, (errs, rates)


@pytest.mark.parametrize("mapping", [0, 1])
def test_sphere_solution_error_is_bounded(oracle_mod, mapping):
    """-omega^2 Delta_S u + u = f with u a degree-2 spherical harmonic, omega^2 = 1,
    f = (1 + 6) u sampled at the centres (nz = 1 uniform: the vertical term is
    zero).  The relative L2 error of the converged multigrid solution stays
    between 1% and 10% for n = 16 .. 64 and does not grow: observed order 0
    (the non-orthogonal grid, see the module docstring)."""
    l, Y = _harmonics()[1]
    errs = []
    for n in (16, 32, 64):
        g = grid(oracle_mod, n, mapping, coarsest_min=4)
        y = Y(g.centres()).reshape(1, 6, n, n)
        u, it, hist = g.mg_solve(g.volumes() * (1 + l * (l + 1)) * y, rtol=1e-12, maxit=100)
        assert hist[-1] <= 1e-12
        area = g.geometry()[0].reshape(1, 6, n, n)
        errs.append(float(np.sqrt((area * (u - y) ** 2).sum() / (area * y ** 2).sum())))
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    print(f"mapping {mapping}: relative L2 error {errs}, observed orders {orders}")
    assert all(0.01 < e < 0.1 for e in errs), errs
    assert errs[2] < 1.1 * errs[0], errs
