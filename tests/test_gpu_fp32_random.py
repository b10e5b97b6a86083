"""FP32 line smoother on fully random iterates at n_z = 128, on the launches that
park the eliminated right-hand side in tensor memory (at least 152 blocks of
128 columns), against the definition of a sweep (Sec. 4.2): u1 = u0 + rho d
with Dtilde d = b - A u0, Dtilde the block (vertical tridiagonal) part of A.

The forward error of an FP32 sweep against the FP64 oracle is not a useful
bar here: the sweep rounds b - A u0, whose vertical terms are up to ~1e10
times the column's diagonal excess on graded columns, and Dtilde^{-1}
amplifies that rounding by the same factor (observed forward errors 1e-2 at
omega^2 = 0.01 and O(1) with strong coupling, while any correct FP32
evaluation may differ from another that much).  What a correct FP32 sweep
does guarantee is a small componentwise backward error: evaluated in FP64,
    |Dtilde d - (b - A u0)| <= C eps32 (|b| + |A||u0| + |Dtilde||d| + |Dtilde||u1|/rho)
(rounding of the residual's terms, of the elimination -- backward stable for
these M-matrices -- of the FP32 coefficients, and of the final update).  The
test checks it element by element with C = 32, for one sweep and for the
second sweep from the first one's FP32 result, and prints the achieved
backward error and the forward error.  A wrong level, neighbour, coefficient
or colour gives an O(1) backward error.  The operator pieces are taken from
the oracle's geometry (areas, transmissibilities, neighbours) and radial
vectors; their sum is checked against the oracle's own A u first.
"""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs
from gpu_util import EPS32, Pair, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# kind, n, nz, graded, omega2, lambda2, smoother
CASES = [
    (1, 64, 128, True, 0.01, 1.0, 0),    # 192 blocks, n % 32 == 0 (aligned staging)
    (1, 80, 128, True, 0.01, 1.0, 0),    # 300 blocks, n % 32 != 0 (neighbour buffer)
    (1, 64, 128, True, 0.01, 1.0, 1),    # block red-black SOR half-sweeps
    (0, 160, 128, True, 0.1, 25.0, 0),   # box, strong vertical coupling (ill-conditioned columns)
]
IDS = ["sph64z128", "sph80z128", "sph64z128rb", "box160z128strong"]
C_BACKWARD = 32.0


@pytest.fixture(scope="module")
def torch_mod():
    return require_gpu()


def f32exact(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


class Pieces:
    """Mass, horizontal and vertical parts of A on level 0 of an oracle grid,
    as (nz, ncol) maps, with their absolute-value counterparts."""

    def __init__(self, og):
        self.og = og
        area, trans, nbr = og.geometry()
        V, G = og.radial()
        w2, l2 = og.omega2, og.lambda2
        self.nz, self.nc = og.nz, og.ncol()
        self.mass = area[None, :] * V[:, None]                      # A_P V_k
        self.tq = w2 * V[:, None, None] * trans[None, :, :]         # w2 V_k T_q  (nz, nc, 4)
        self.nbr = nbr
        self.gu = w2 * l2 * area[None, :] * G[1:, None]             # coupling to k+1
        self.gd = w2 * l2 * area[None, :] * G[:-1, None]            # coupling to k-1

    def _shift(self, x):
        up = np.zeros_like(x)
        dn = np.zeros_like(x)
        up[:-1] = x[1:]
        dn[1:] = x[:-1]
        return up, dn

    def diag_block(self, x, absolute=False):
        """Dtilde x (or |Dtilde| |x|): mass, the diagonal of the horizontal part
        and the vertical part."""
        up, dn = self._shift(x)
        hd = self.tq.sum(axis=2)
        if absolute:
            x, up, dn = np.abs(x), np.abs(up), np.abs(dn)
            return (self.mass + hd) * x + self.gu * (x + up) + self.gd * (x + dn)
        return (self.mass + hd) * x + self.gu * (x - up) + self.gd * (x - dn)

    def apply(self, x, absolute=False):
        """A x (or |A| |x|)."""
        nb = x[:, self.nbr]                                          # (nz, nc, 4)
        if absolute:
            return self.diag_block(x, True) + (self.tq * np.abs(nb)).sum(axis=2)
        return self.diag_block(x) - (self.tq * nb).sum(axis=2)


def backward_error(pc, b, u0, u1, rho, cols=None):
    """Largest componentwise backward error of the sweep u0 -> u1, over the
    updated columns `cols` (all when None), in units of eps32."""
    d = (u1 - u0) / rho
    lhs = pc.diag_block(d) - (b - pc.apply(u0))
    bound = (np.abs(b) + pc.apply(u0, True) + pc.diag_block(d, True) +
             pc.diag_block(u1, True) / rho)
    ratio = np.abs(lhs) / bound / EPS32
    if cols is not None:
        ratio = ratio[:, cols]
    return float(ratio.max())


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp32_smoother_random_iterate(torch_mod, oracle_mod, case):
    kind, n, nz, graded, w2, l2, smoother = case
    p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, precision=1,
             smoother=smoother)
    nc = p.og.ncol()
    assert (nc + 127) // 128 >= 152  # the tensor-memory launch
    pc = Pieces(p.og)
    sh = p.og.shape()
    u0 = f32exact(inputs.uniform_pm1(sh, member=501)).reshape(nz, nc)
    b = f32exact(p.og.volumes() * inputs.uniform_pm1(sh, member=502)).reshape(nz, nc)
    # the test's operator pieces are the oracle's operator
    assert rel_l2(pc.apply(u0), p.og.apply(u0).reshape(nz, nc)) <= 1e-13
    rho = 1.0 if smoother == 1 else 0.8
    bd = p.dev(b.reshape(sh), True)
    ud = p.dev(u0.reshape(sh), True)
    iters = [u0]
    for sweep in range(2):
        p.sv.level_smooth(0, bd, ud, nsweeps=1, rho=rho, fp32=True)
        iters.append(p.host(ud).reshape(nz, nc))
    worst = 0.0
    for s in range(2):
        ua, ub = iters[s], iters[s + 1]
        if smoother == 0:
            worst = max(worst, backward_error(pc, b, ua, ub, rho))
        else:
            # red columns from ua, then black columns from the half-swept iterate
            red = p.og.colour() == 0
            mid = np.where(red[None, :], ub, ua)
            worst = max(worst, backward_error(pc, b, ua, mid, rho, cols=red))
            worst = max(worst, backward_error(pc, b, mid, ub, rho, cols=~red))
    fwd_ref = (p.og.smooth(b.reshape(sh), u0.reshape(sh), 2, rho) if smoother == 0 else None)
    fwd = rel_l2(iters[2], fwd_ref) if fwd_ref is not None else float("nan")
    print(f"{n}x{n}x{nz} smoother {smoother}: componentwise backward error {worst:.2f} eps32 "
          f"(bar {C_BACKWARD:.0f}), forward error of two sweeps against the oracle {fwd:.2e}")
    assert worst <= C_BACKWARD


# Levels of at most 9,728 columns take the partitioned line solve (eight
# segments per column joined by a system on the seven levels between them):
# the same backward-error bar, and the whole-column elimination
# (line_part = 0) beside it for reference.
PART_CASES = [
    (1, 32, 128, True, 0.01, 1.0, 0),    # 6144 columns, n % 32 == 0
    (1, 40, 64, True, 0.01, 1.0, 0),     # 9600 columns, n % 32 != 0 (neighbour buffer)
    (1, 32, 128, True, 0.01, 1.0, 1),    # block red-black SOR half-sweeps
    (0, 96, 128, True, 0.1, 25.0, 0),    # box, strong vertical coupling
    (1, 16, 256, True, 0.01, 1.0, 0),    # n_z = 256: segments of 31 levels
    (0, 8, 16, False, 0.01, 1.0, 0),     # n_z = 16: segments of one level
]
PART_IDS = ["sph32z128", "sph40z64", "sph32z128rb", "box96z128strong", "sph16z256", "box8z16"]


@pytest.mark.parametrize("case", PART_CASES, ids=PART_IDS)
def test_fp32_partitioned_smoother_random_iterate(torch_mod, oracle_mod, case):
    kind, n, nz, graded, w2, l2, smoother = case
    worst = {}
    for line_part in (1, 0):
        p = Pair(oracle_mod, kind, n, nz, omega2=w2, lambda2=l2, graded=graded, precision=1,
                 smoother=smoother, line_part=line_part)
        nc = p.og.ncol()
        assert nc <= 9728
        pc = Pieces(p.og)
        sh = p.og.shape()
        u0 = f32exact(inputs.uniform_pm1(sh, member=511)).reshape(nz, nc)
        b = f32exact(p.og.volumes() * inputs.uniform_pm1(sh, member=512)).reshape(nz, nc)
        rho = 1.0 if smoother == 1 else 0.8
        bd = p.dev(b.reshape(sh), True)
        ud = p.dev(u0.reshape(sh), True)
        iters = [u0]
        for sweep in range(2):
            p.sv.level_smooth(0, bd, ud, nsweeps=1, rho=rho, fp32=True)
            iters.append(p.host(ud).reshape(nz, nc))
        w = 0.0
        for s in range(2):
            ua, ub = iters[s], iters[s + 1]
            if smoother == 0:
                w = max(w, backward_error(pc, b, ua, ub, rho))
            else:
                red = p.og.colour() == 0
                mid = np.where(red[None, :], ub, ua)
                w = max(w, backward_error(pc, b, ua, mid, rho, cols=red))
                w = max(w, backward_error(pc, b, mid, ub, rho, cols=~red))
        worst[line_part] = w
    print(f"{n}x{n}x{nz} smoother {smoother}: componentwise backward error, partitioned "
          f"{worst[1]:.2f} eps32, whole column {worst[0]:.2f} eps32 (bar {C_BACKWARD:.0f})")
    assert worst[1] <= C_BACKWARD and worst[0] <= C_BACKWARD
