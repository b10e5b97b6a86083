"""Pins against numbers printed in the paper (CPU only).

tests/golden/table1_parameter_space.txt holds Table 1 of arXiv:1307.2036.
omega^2 and lambda^2 follow from Eq. omega2lambda2 and the time step; the
anisotropy beta = lambda^2 (dx/dz)^2 follows from the typical spacing
dx = 2 pi R / (4 nx) (Sec. 3.1.2) and the level spacing of Eq. VerticalGrading,
which the input generator's radial_levels() produces.  Every printed entry is
reproduced to 1% except beta_top of the nx = 512 row, printed as 4.69 where the
paper's own formulas give 46.9 (read as a misprint by a factor of ten).
"""
import os

import numpy as np

from paper_1307_2036_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_parameter_space.txt")
R_EARTH = 6.371e6
C_H, N_BUOY, ALPHA = 550.0, 0.018, 0.5


def load():
    return np.loadtxt(GOLDEN, comments="#")


def test_omega2_lambda2_from_time_step():
    for nx, dx_km, dt, w2, l2, *_ in load():
        omega2 = (ALPHA * C_H * dt / R_EARTH) ** 2
        lambda2 = 1.0 / (1.0 + (ALPHA * dt) ** 2 * N_BUOY ** 2)
        assert abs(omega2 / w2 - 1) < 0.01, (nx, omega2, w2)
        assert abs(lambda2 / l2 - 1) < 0.01, (nx, lambda2, l2)
        assert abs(2 * np.pi * R_EARTH / (4 * nx) / (dx_km * 1e3) - 1) < 0.02


def test_anisotropy_from_vertical_grading():
    nz = 128
    r = inputs.radial_levels(nz, H=0.01, graded=True)
    dz = np.diff(r) * R_EARTH
    for nx, dx_km, dt, w2, l2, bb, bm, bt in load():
        dx = 2 * np.pi * R_EARTH / (4 * nx)
        lambda2 = 1.0 / (1.0 + (ALPHA * dt) ** 2 * N_BUOY ** 2)
        beta = lambda2 * (dx / dz[[0, nz // 2, nz - 1]]) ** 2
        printed = np.array([bb, bm, bt])
        if nx == 512:
            printed[2] *= 10.0  # misprint in the table
        assert np.all(np.abs(beta / printed - 1) < 0.01), (nx, beta, printed)


def test_horizontal_coupling_value():
    """Sec. 3.1.2: nx = 256, dt = 10 min gives C_horiz = alpha^2 (c_h dt / dx)^2 ~ 17.8."""
    dx = 2 * np.pi * R_EARTH / (4 * 256)
    assert abs(ALPHA ** 2 * (C_H * 600.0 / dx) ** 2 - 17.8) < 0.1
