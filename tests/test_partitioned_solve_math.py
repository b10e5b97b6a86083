"""The mathematics of the partitioned line solve (the small levels' line
smoother, opts.line_part = 1), restated here in numpy and checked against the
oracle's whole-column elimination (Algorithm Thomas in the excess form).

A column's rows are  -lo_k e_{k-1} + (lo_k + hi_k + X_k) e_k - hi_k e_{k+1} = r_k
with X_k > 0.  The nz levels form eight ranges of nz / 8; the last level of
ranges 0..6 is a separator, the others a segment.  Each segment is eliminated
with its couplings to the separators on the right-hand side, for four
right-hand sides: r (y), a unit value at the separator below (alpha) and above
(beta), and the segment's excess X (z = 1 - alpha - beta, formed directly).
The separators satisfy a tridiagonal system with off-diagonals lo_q alpha and
hi_q beta of the adjoining segments and excess X_q + lo_q z_below +
hi_q z_above; every level is then y + alpha e_below + beta e_above.

Checked: in FP64 the result is the oracle's solution to rounding (a wrong sign,
index or coefficient in the joining system fails that); in FP32, on graded
columns whose coupling is up to 1e13 times the excess, its forward error stays
at the level of the FP32 whole-column elimination's (both below 1e-4, the
columns' conditioning), while the same joining system with its diagonal formed
by subtraction (D_q - lo_q beta_below - hi_q alpha_above, the textbook Schur
complement) loses two digits at 1e10 and every digit at 1e13.
"""
import numpy as np
import pytest

import oracle


def excess_thomas(lo, hi, X, r, dt):
    """Whole-column elimination in the excess form, in precision dt."""
    n = len(r)
    cp = np.zeros(n, dt)
    fp = np.zeros(n, dt)
    ratio, prev = dt(0), dt(0)
    for k in range(n):
        E = dt(X[k] + lo[k] * ratio)
        inv = dt(1) / dt(E + hi[k])
        cp[k] = hi[k] * inv
        fp[k] = dt(r[k] + lo[k] * prev) * inv
        ratio, prev = dt(E * inv), fp[k]
    e = np.zeros(n, dt)
    e[-1] = fp[-1]
    for k in range(n - 2, -1, -1):
        e[k] = dt(fp[k] + cp[k] * e[k + 1])
    return e


def partitioned(lo, hi, X, r, dt, ranges=8, subtractive=False):
    lo, hi, X, r = (np.asarray(v, dt) for v in (lo, hi, X, r))
    n = len(r)
    Ls = n // ranges
    seps = [(w + 1) * Ls - 1 for w in range(ranges - 1)]
    segs = []
    for w in range(ranges):
        a, b = w * Ls, (seps[w] if w < ranges - 1 else n)
        L = b - a
        cp, fy, fa, fz = (np.zeros(L, dt) for _ in range(4))
        ratio, py, pa, pz = dt(1), dt(0), dt(1), dt(0)   # rho = 1 at a segment's start
        for i in range(L):
            k = a + i
            E = dt(X[k] + lo[k] * ratio)
            inv = dt(1) / dt(E + hi[k])
            ratio = dt(E * inv)
            cp[i] = hi[k] * inv
            py = fy[i] = dt(r[k] + lo[k] * py) * inv
            pa = fa[i] = dt(lo[k] * pa) * inv
            pz = fz[i] = dt(X[k] + lo[k] * pz) * inv
        y, al, be, z = (np.zeros(L, dt) for _ in range(4))
        ny, na, nb, nzv = dt(0), dt(0), dt(1), dt(0)
        for i in range(L - 1, -1, -1):
            ny = y[i] = dt(fy[i] + cp[i] * ny)
            na = al[i] = dt(fa[i] + cp[i] * na)
            nzv = z[i] = dt(fz[i] + cp[i] * nzv)
            nb = be[i] = dt(cp[i] * nb)
        segs.append((a, b, y, al, be, z))
    S = ranges - 1
    slo, shi, sX, sr = (np.zeros(S, dt) for _ in range(4))
    for w, q in enumerate(seps):
        _, _, yL, aL, bL, zL = segs[w]
        _, _, yR, aR, bR, zR = segs[w + 1]
        slo[w] = lo[q] * aL[-1]
        shi[w] = hi[q] * bR[0]
        if subtractive:   # diagonal by subtraction, excess = diagonal - couplings
            D = dt(lo[q] + hi[q] + X[q])
            diag = dt(dt(D - lo[q] * bL[-1]) - hi[q] * aR[0])
            sX[w] = dt(dt(diag - slo[w]) - shi[w])
        else:
            sX[w] = dt(dt(X[q] + lo[q] * zL[-1]) + hi[q] * zR[0])
        sr[w] = dt(dt(r[q] + lo[q] * yL[-1]) + hi[q] * yR[0])
    es = excess_thomas(slo, shi, sX, sr, dt)
    e = np.zeros(n, dt)
    for w, (a, b, y, al, be, z) in enumerate(segs):
        eb = es[w - 1] if w > 0 else dt(0)
        ea = es[w] if w < S else dt(0)
        e[a:b] = y + al * eb + be * ea
    for w, q in enumerate(seps):
        e[q] = es[w]
    return e


def graded_column(nz, ratio, seed):
    rng = np.random.default_rng(seed)
    t = np.arange(nz + 1) / nz
    rl = 1 + 0.01 * t * t
    dr = np.diff(rl)
    g = np.zeros(nz + 1)
    g[1:-1] = 1.0 / (0.5 * (dr[1:] + dr[:-1]))
    g *= ratio / g[1:-1].max()
    X = dr / dr.max()
    return g[:-1].copy(), g[1:].copy(), X, rng.uniform(-1, 1, nz)


@pytest.mark.parametrize("nz", [16, 64, 128, 256])
@pytest.mark.parametrize("ratio", [1e2, 1e8, 1e13])
def test_fp64_partitioned_is_the_thomas_solution(nz, ratio):
    lo, hi, X, r = graded_column(nz, ratio, seed=nz)
    ref = oracle.thomas_excess(X, hi, lo, r)
    e = partitioned(lo, hi, X, r, np.float64)
    assert np.linalg.norm(e - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("nz", [128, 256])
@pytest.mark.parametrize("ratio", [1e2, 1e6, 1e10, 1e13])
def test_fp32_partitioned_keeps_the_excess_form_accuracy(nz, ratio):
    lo, hi, X, r = graded_column(nz, ratio, seed=7 * nz)
    ref = oracle.thomas_excess(X, hi, lo, r)
    nrm = np.linalg.norm(ref)
    err = lambda e: np.linalg.norm(e.astype(np.float64) - ref) / nrm
    whole = err(excess_thomas(lo.astype(np.float32), hi.astype(np.float32),
                              X.astype(np.float32), r.astype(np.float32), np.float32))
    part = err(partitioned(lo, hi, X, r, np.float32))
    sub = err(partitioned(lo, hi, X, r, np.float32, subtractive=True))
    print(f"nz {nz}, coupling/excess {ratio:.0e}: FP32 forward error whole column "
          f"{whole:.1e}, partitioned {part:.1e}, partitioned with a subtracted diagonal {sub:.1e}")
    # both at the level the columns' conditioning sets in FP32 (observed
    # 3e-7 .. 2e-5 for either, varying with the right-hand side's rounding)
    assert whole <= 1e-4 and part <= 1e-4
    if ratio >= 1e10:
        assert not (sub <= 1e-2)   # the subtraction loses the excess entirely
