"""Pins of the oracle's grid geometry and connectivity (CPU only).

Each check uses a fact that the oracle's code does not itself compute:
  * the sphere has area 4 pi, and the exact area of a gnomonic coordinate
    rectangle, F(x, y) = atan(x y / sqrt(1 + x^2 + y^2)) summed over the corners
    (the oracle uses spherical-triangle solid angles instead);
  * gnomonic grid lines are great circles, so the faces along one grid line add
    up to that line's whole arc;
  * two cells are neighbours exactly when they share a face: the end points of
    the face seen from either side coincide on the sphere;
  * rediscretised coarse cells are the unions of their four children.
Grid: Eqs. x1x2_1/x1x2_2 (cubed sphere), Sec. 3.1; periodic box of side 2 pi.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs

# Panel frames (normal N, axes A, B with A x B = N): the numbering convention of
# the cell index c = (p n + j) n + i, shared by the oracle and the library as a
# data-layout definition.
N_ = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
A_ = np.array([[0, 1, 0], [-1, 0, 0], [0, -1, 0], [1, 0, 0], [0, 1, 0], [0, 1, 0]], float)
B_ = np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1], [-1, 0, 0], [1, 0, 0]], float)


def mapcoord(t, n, mapping):
    t = np.asarray(t, float)
    if mapping == 1:
        return -1.0 + 2.0 * t / n
    return np.tan(-np.pi / 4 + t * (np.pi / 2) / n)


def corners(n, mapping):
    """unit vectors of the four corners of every cell, shape (6, n, n, 4, 3),
    corner order (i, j), (i+1, j), (i, j+1), (i+1, j+1)."""
    t = mapcoord(np.arange(n + 1), n, mapping)
    out = np.empty((6, n, n, 4, 3))
    for p in range(6):
        X = (N_[p][None, None, :] + t[None, :, None] * A_[p][None, None, :] +
             t[:, None, None] * B_[p][None, None, :])  # [j, i, 3]
        X /= np.linalg.norm(X, axis=-1, keepdims=True)
        out[p, :, :, 0] = X[:-1, :-1]
        out[p, :, :, 1] = X[:-1, 1:]
        out[p, :, :, 2] = X[1:, :-1]
        out[p, :, :, 3] = X[1:, 1:]
    return out


def sphere(oracle_mod, n, mapping=0, nz=2):
    return oracle_mod.Grid(1, n, nz, inputs.radial_levels(nz), 0.01, 1.0, mapping=mapping,
                           coarsest_min=1)


@pytest.mark.parametrize("mapping", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 8, 32])
def test_sphere_total_area_is_4pi(oracle_mod, n, mapping):
    g = sphere(oracle_mod, n, mapping)
    area, _, _ = g.geometry()
    assert abs(area.sum() - 4 * np.pi) < 1e-13


@pytest.mark.parametrize("mapping", [0, 1])
def test_sphere_cell_area_closed_form(oracle_mod, mapping):
    n = 12
    g = sphere(oracle_mod, n, mapping)
    area, _, _ = g.geometry()
    t = mapcoord(np.arange(n + 1), n, mapping)
    F = np.arctan(t[None, :] * t[:, None] / np.sqrt(1 + t[None, :] ** 2 + t[:, None] ** 2))
    cell = F[1:, 1:] - F[1:, :-1] - F[:-1, 1:] + F[:-1, :-1]  # [j, i]
    expect = np.broadcast_to(cell, (6, n, n)).reshape(-1)
    assert np.max(np.abs(area - expect) / expect) < 1e-12


@pytest.mark.parametrize("mapping", [0, 1])
def test_face_lengths_add_up_along_grid_lines(oracle_mod, mapping):
    n = 10
    g = sphere(oracle_mod, n, mapping)
    ell, _ = g.face_lengths()
    ell = ell.reshape(6, n, n, 4)
    t = mapcoord(np.arange(n + 1), n, mapping)
    for p in range(6):
        for i in range(n + 1):
            # the line xi = t_i runs from eta = -1 to eta = 1 on a great circle
            a = N_[p] + t[i] * A_[p] - B_[p]
            b = N_[p] + t[i] * A_[p] + B_[p]
            whole = np.arccos(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b))
            segs = ell[p, :, i, 0].sum() if i < n else ell[p, :, n - 1, 1].sum()
            assert abs(segs - whole) < 1e-13
    # the panel boundary is the cube edge: arc acos(1/3)
    assert abs(ell[0, :, 0, 0].sum() - np.arccos(1.0 / 3.0)) < 1e-13


@pytest.mark.parametrize("mapping", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_sphere_neighbours_share_a_face(oracle_mod, n, mapping):
    g = sphere(oracle_mod, n, mapping)
    _, _, nbr = g.geometry()
    C = corners(n, mapping).reshape(-1, 4, 3)
    face_corners = {0: (0, 2), 1: (1, 3), 2: (0, 1), 3: (2, 3)}
    ncol = 6 * n * n
    for c in range(ncol):
        assert len(set(nbr[c])) == (4 if n > 1 else 4)
        for q in range(4):
            Q = nbr[c, q]
            assert 0 <= Q < ncol and Q != c
            mine = C[c, list(face_corners[q])]
            # some face of Q has the same two end points
            found = False
            for qq in range(4):
                theirs = C[Q, list(face_corners[qq])]
                d1 = np.abs(mine - theirs).max()
                d2 = np.abs(mine - theirs[::-1]).max()
                if min(d1, d2) < 1e-12:
                    found = True
                    assert nbr[Q, qq] == c  # and Q points back across it
            assert found, (c, q, Q)


def test_sphere_face_data_symmetric(oracle_mod):
    n = 16
    g = sphere(oracle_mod, n, 0)
    _, trans, nbr = g.geometry()
    ell, dist = g.face_lengths()
    for c in range(6 * n * n):
        for q in range(4):
            Q = nbr[c, q]
            qq = int(np.where(nbr[Q] == c)[0][0])
            assert abs(ell[c, q] - ell[Q, qq]) < 1e-14
            assert abs(dist[c, q] - dist[Q, qq]) < 1e-14
            assert abs(trans[c, q] - trans[Q, qq]) < 1e-12


@pytest.mark.parametrize("mapping", [0, 1])
def test_coarse_cells_are_unions_of_children(oracle_mod, mapping):
    n = 16
    g = oracle_mod.Grid(1, n, 2, inputs.radial_levels(2), 0.01, 1.0, mapping=mapping,
                        coarsest_min=2)
    assert g.nlevels == 4
    for lev in range(g.nlevels - 1):
        nf = g.level_n(lev)
        af = g.geometry(lev)[0].reshape(6, nf // 2, 2, nf // 2, 2)
        ac = g.geometry(lev + 1)[0].reshape(6, nf // 2, nf // 2)
        assert np.max(np.abs(af.sum(axis=(2, 4)) - ac) / ac) < 1e-12
        ef = g.face_lengths(lev)[0].reshape(6, nf // 2, 2, nf // 2, 2, 4)
        ec = g.face_lengths(lev + 1)[0].reshape(6, nf // 2, nf // 2, 4)
        west = ef[:, :, :, :, 0, 0].sum(axis=2)  # children with i even, face -i
        south = ef[:, :, 0, :, :, 2].sum(axis=3)  # children with j even, face -j
        assert np.max(np.abs(west - ec[..., 0]) / ec[..., 0]) < 1e-12
        assert np.max(np.abs(south - ec[..., 2]) / ec[..., 2]) < 1e-12


def test_box_geometry(oracle_mod):
    n = 6
    g = oracle_mod.Grid(0, n, 3, inputs.radial_levels(3), 0.01, 1.0)
    area, trans, nbr = g.geometry()
    h = 2 * np.pi / n
    assert np.allclose(area, h * h, rtol=1e-15)
    assert np.allclose(trans, 1.0, rtol=1e-15)
    for j in range(n):
        for i in range(n):
            c = j * n + i
            assert list(nbr[c]) == [j * n + (i - 1) % n, j * n + (i + 1) % n,
                                    ((j - 1) % n) * n + i, ((j + 1) % n) * n + i]


def test_hierarchy_sizes(oracle_mod):
    cases = {(0, 32): [32, 16, 8, 4], (0, 256): [256, 128, 64, 32, 16, 8, 4],
             (1, 48): [48, 24, 12, 6], (1, 6): [6], (1, 384): [384, 192, 96, 48, 24, 12, 6]}
    for (kind, n), sizes in cases.items():
        g = oracle_mod.Grid(kind, n, 2, inputs.radial_levels(2), 0.01, 1.0)
        assert [g.level_n(l) for l in range(g.nlevels)] == sizes


def test_radial_metric_terms(oracle_mod):
    """V_k is the volume integral of r^2 (checked with Simpson's rule, exact for
    quadratics); G_k vanishes at the two Neumann boundaries."""
    nz = 16
    r = inputs.radial_levels(nz, graded=True)
    g = oracle_mod.Grid(0, 4, nz, r, 0.01, 1.0)
    V, G = g.radial()
    mid = 0.5 * (r[1:] + r[:-1])
    simpson = (r[1:] - r[:-1]) / 6.0 * (r[:-1] ** 2 + 4 * mid ** 2 + r[1:] ** 2)
    assert np.max(np.abs(V - simpson) / V) < 1e-12
    assert G[0] == 0.0 and G[nz] == 0.0
    assert np.all(G[1:nz] > 0)
    # total volume of the shell over the unit sphere: ((1+H)^3 - 1) / 3
    assert abs(V.sum() - ((1.01) ** 3 - 1) / 3) < 1e-15
