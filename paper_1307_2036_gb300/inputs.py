"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the solver: it draws right-hand sides,
radial level sets and per-member parameters from a counter-based generator, so
every value depends only on (seed, member, global cell id) and not on batching
or on the device.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a hash of a counter.
Uniform[-1, 1): 2 * (x >> 11) * 2^-53 - 1.  N(0, 1): Box-Muller on two
uniforms drawn from counters 2 id and 2 id + 1.

Array shape convention: (nz, P, n, n), vertical index slowest; the global cell
id of (k, p, j, i) is ((k P + p) n + j) n + i.
"""
import numpy as np

DEFAULT_SEED = 20130708
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z):
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _key(seed, member, stream):
    with np.errstate(over="ignore"):
        s = _mix(np.array([seed], dtype=np.uint64) + _GOLDEN)
        s = _mix(s ^ (np.uint64(member) * _GOLDEN + np.uint64(1)))
        s = _mix(s ^ (np.uint64(stream) * _M1 + np.uint64(7)))
    return s[0]


def _bits(seed, member, stream, counters):
    key = _key(seed, member, stream)
    with np.errstate(over="ignore"):
        return _mix(key + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN)


def _unit(bits):
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(shape, seed=DEFAULT_SEED, member=0, chunk=1 << 24):
    """i.i.d. uniform[-1, 1) values, one per cell id."""
    total = int(np.prod(shape))
    out = np.empty(total, dtype=np.float64)
    for s in range(0, total, chunk):
        ids = np.arange(s, min(total, s + chunk), dtype=np.uint64)
        out[s:s + len(ids)] = 2.0 * _unit(_bits(seed, member, 1, ids)) - 1.0
    return out.reshape(shape)


def gaussian(shape, seed=DEFAULT_SEED, member=0, chunk=1 << 23):
    """i.i.d. N(0, 1) values (Box-Muller), one per cell id."""
    total = int(np.prod(shape))
    out = np.empty(total, dtype=np.float64)
    for s in range(0, total, chunk):
        ids = np.arange(s, min(total, s + chunk), dtype=np.uint64)
        u1 = _unit(_bits(seed, member, 2, 2 * ids))
        u2 = _unit(_bits(seed, member, 2, 2 * ids + np.uint64(1)))
        out[s:s + len(ids)] = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    return out.reshape(shape)


def smooth_per_panel(f, sweeps=3):
    """`sweeps` passes of f <- f/2 + (sum of the four in-panel neighbours)/8 on
    every vertical level and panel; across a panel edge (or the box edge) the
    missing neighbour is replaced by the cell itself.  f: (nz, P, n, n)."""
    f = np.array(f, dtype=np.float64, copy=True)
    for _ in range(sweeps):
        g = np.pad(f, ((0, 0), (0, 0), (1, 1), (1, 1)), mode="edge")
        f = 0.5 * f + 0.125 * (g[:, :, 1:-1, :-2] + g[:, :, 1:-1, 2:] + g[:, :, :-2, 1:-1] +
                               g[:, :, 2:, 1:-1])
    return f


def radial_levels(nz, H=0.01, graded=False):
    """nz+1 radii on [1, 1+H]: uniform, or r_k = 1 + H (k/nz)^2 (Eq. VerticalGrading)."""
    t = np.arange(nz + 1, dtype=np.float64) / nz
    return 1.0 + H * (t * t if graded else t)


def fourier_cos_mode(n, nz, kx=3, ky=5, m=2, side=2 * np.pi):
    """f = cos(kx x_i + ky y_j) cos(pi m (k + 1/2) / nz) on the n x n periodic box,
    x_i = (i + 1/2) h, h = side / n.  Shape (nz, 1, n, n)."""
    h = side / n
    x = (np.arange(n) + 0.5) * h
    horiz = np.cos(kx * x[None, :] + ky * x[:, None])  # [j, i]
    vert = np.cos(np.pi * m * (np.arange(nz) + 0.5) / nz)
    return (vert[:, None, None, None] * horiz[None, None, :, :]).copy()


def member_params(count, seed=DEFAULT_SEED, omega2_range=(1e-3, 1e-1), lam_range=(0.5, 5.0)):
    """Per-member (omega^2, lambda): omega^2 log-uniform, lambda uniform."""
    ids = np.arange(count, dtype=np.uint64)
    u1 = _unit(_bits(seed, 0, 3, 2 * ids))
    u2 = _unit(_bits(seed, 0, 3, 2 * ids + np.uint64(1)))
    lo, hi = np.log(omega2_range[0]), np.log(omega2_range[1])
    omega2 = np.exp(lo + (hi - lo) * u1)
    lam = lam_range[0] + (lam_range[1] - lam_range[0]) * u2
    return omega2, lam


def request_stream(count, rate=200.0, seed=DEFAULT_SEED, sizes=(48, 96, 192, 384),
                   nzs=(32, 64, 128), tols=(1e-5, 1e-10)):
    """Serving workload: Poisson arrival times (mean rate `rate` per second) and,
    per request, panel size n, nz, omega^2, lambda and tolerance, all uniform over
    the listed choices (omega^2, lambda as in member_params)."""
    ids = np.arange(count, dtype=np.uint64)
    gaps = -np.log1p(-_unit(_bits(seed, 0, 4, ids))) / rate
    arrivals = np.cumsum(gaps)
    pick = lambda stream, choices: np.asarray(choices)[
        np.minimum((_unit(_bits(seed, 0, stream, ids)) * len(choices)).astype(np.int64),
                   len(choices) - 1)]
    n = pick(5, sizes)
    nz = pick(6, nzs)
    tol = pick(7, tols)
    omega2, lam = member_params(count, seed=seed + 1)
    return {"arrival": arrivals, "n": n, "nz": nz, "tol": tol, "omega2": omega2, "lam": lam}
