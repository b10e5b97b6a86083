"""ellsolve oracle: plain FP64 CPU reference of the discretisation and solvers of
Mueller & Scheichl, arXiv:1307.2036 (C code in ellsolve_oracle.c, loaded here
through ctypes).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  It shares
no code with the CUDA library and never consumes its output.

Arrays are numpy float64 with shape (nz, P, n, n) (vertical index slowest).
"""
import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        lp = C.POINTER(C.c_long)
        vp = C.c_void_p
        sig = {
            "og_create": (vp, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_double,
                               C.c_double, C.c_int, C.c_int]),
            "og_destroy": (None, [vp]),
            "og_nlevels": (C.c_int, [vp]),
            "og_npanel": (C.c_int, [vp]),
            "og_level_n": (C.c_int, [vp, C.c_int]),
            "og_level_ncol": (C.c_long, [vp, C.c_int]),
            "og_get_geometry": (None, [vp, C.c_int, dp, dp, lp]),
            "og_get_centres": (None, [vp, C.c_int, dp]),
            "og_get_face_lengths": (None, [vp, C.c_int, dp, dp]),
            "og_get_radial": (None, [vp, dp, dp]),
            "og_volumes": (None, [vp, C.c_int, dp]),
            "og_apply": (None, [vp, C.c_int, dp, dp]),
            "og_residual": (None, [vp, C.c_int, dp, dp, dp]),
            "og_assemble_dense": (None, [vp, C.c_int, dp]),
            "og_thomas_paper": (None, [C.c_int, dp, dp, dp, dp, dp]),
            "og_thomas_excess": (None, [C.c_int, dp, dp, dp, dp, dp]),
            "og_smooth": (None, [vp, C.c_int, dp, dp, C.c_int, C.c_double]),
            "og_line_precond": (None, [vp, C.c_int, dp, dp]),
            "og_smooth_rb": (None, [vp, C.c_int, dp, dp, C.c_int, C.c_double]),
            "og_rb_ssor": (None, [vp, C.c_int, dp, dp, C.c_double]),
            "og_set_smoother": (None, [vp, C.c_int]),
            "og_set_precond": (None, [vp, C.c_int, C.c_double]),
            "og_set_profiles": (None, [vp, dp, dp]),
            "og_set_mg_precond": (None, [vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int]),
            "og_set_fmg": (None, [vp, C.c_int]),
            "og_fmg": (None, [vp, dp, dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                              C.c_int]),
            "og_restrict": (None, [vp, C.c_int, dp, dp]),
            "og_prolong_add": (None, [vp, C.c_int, dp, dp, C.c_int]),
            "og_vcycle": (None, [vp, dp, dp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                 C.c_int]),
            "og_mg_solve": (C.c_int, [vp, dp, dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_double, C.c_double, C.c_int, dp]),
            "og_pcg_solve": (C.c_int, [vp, dp, dp, C.c_double, C.c_int, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def thomas_paper(a, b, c, f):
    """Algorithm Thomas as printed (a diagonal, b super-, c sub-diagonal)."""
    a, b, c, f = (_f64(x) for x in (a, b, c, f))
    u = np.empty_like(f)
    _load().og_thomas_paper(len(f), _dp(a), _dp(b), _dp(c), _dp(f), _dp(u))
    return u


def thomas_excess(delta, up, lo, f):
    """Algorithm Thomas for diag = delta + up + lo, super = -up, sub = -lo."""
    delta, up, lo, f = (_f64(x) for x in (delta, up, lo, f))
    u = np.empty_like(f)
    _load().og_thomas_excess(len(f), _dp(delta), _dp(up), _dp(lo), _dp(f), _dp(u))
    return u


class Grid:
    """One discretised problem: grid, radial levels, omega^2, lambda^2 and the
    horizontal multigrid hierarchy (level 0 finest)."""

    def __init__(self, kind, n, nz, r, omega2, lambda2, mapping=0, side=2 * np.pi,
                 coarsest_min=4, max_levels=0, smoother=0, precond=0, precond_rho=1.0,
                 p_cell=None, q_face=None, mg_precond=None, fmg=False):
        """smoother: 0 block Jacobi, 1 block red-black SOR (smooth, vcycle,
        mg_solve); precond: 0 block Jacobi, 1 block red-black SSOR, 2 one V-cycle
        (pcg_solve; mg_precond = (nu_pre, nu_post, nu_coarse, rho, prolong));
        p_cell[nz], q_face[nz+1]: vertical background profiles (V_k and G_k
        multipliers), None: the model equation; fmg: the first cycle of
        mg_solve and the V-cycle preconditioner are full multigrid cycles."""
        lib = _load()
        r = _f64(r)
        assert r.shape == (nz + 1,)
        self.kind, self.n, self.nz, self.mapping = kind, n, nz, mapping
        self.omega2, self.lambda2 = omega2, lambda2
        self._h = lib.og_create(kind, n, nz, mapping, side, _dp(r), omega2, lambda2,
                                coarsest_min, max_levels)
        lib.og_set_smoother(self._h, smoother)
        if p_cell is not None or q_face is not None:
            pc = _f64(np.ones(nz) if p_cell is None else p_cell)
            qf = _f64(np.ones(nz + 1) if q_face is None else q_face)
            assert pc.shape == (nz,) and qf.shape == (nz + 1,)
            lib.og_set_profiles(self._h, _dp(pc), _dp(qf))
        lib.og_set_precond(self._h, precond, precond_rho)
        if mg_precond is not None:
            lib.og_set_mg_precond(self._h, *mg_precond)
        lib.og_set_fmg(self._h, 1 if fmg else 0)
        self.P = lib.og_npanel(self._h)
        self.nlevels = lib.og_nlevels(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.og_destroy(self._h)
            self._h = None

    # -- shapes -----------------------------------------------------------
    def level_n(self, lev=0):
        return _load().og_level_n(self._h, lev)

    def ncol(self, lev=0):
        return _load().og_level_ncol(self._h, lev)

    def shape(self, lev=0):
        n = self.level_n(lev)
        return (self.nz, self.P, n, n)

    def zeros(self, lev=0):
        return np.zeros(self.shape(lev))

    # -- geometry ---------------------------------------------------------
    def geometry(self, lev=0):
        nc = self.ncol(lev)
        area = np.empty(nc)
        trans = np.empty((nc, 4))
        nbr = np.empty((nc, 4), dtype=np.int64)
        _load().og_get_geometry(self._h, lev, _dp(area), _dp(trans),
                                nbr.ctypes.data_as(C.POINTER(C.c_long)))
        return area, trans, nbr

    def centres(self, lev=0):
        xyz = np.empty((self.ncol(lev), 3))
        _load().og_get_centres(self._h, lev, _dp(xyz))
        return xyz

    def face_lengths(self, lev=0):
        nc = self.ncol(lev)
        ell, dist = np.empty((nc, 4)), np.empty((nc, 4))
        _load().og_get_face_lengths(self._h, lev, _dp(ell), _dp(dist))
        return ell, dist

    def radial(self):
        V, G = np.empty(self.nz), np.empty(self.nz + 1)
        _load().og_get_radial(self._h, _dp(V), _dp(G))
        return V, G

    def volumes(self, lev=0):
        v = np.empty(self.shape(lev))
        _load().og_volumes(self._h, lev, _dp(v))
        return v

    # -- operator ---------------------------------------------------------
    def apply(self, u, lev=0):
        u = _f64(u).reshape(self.shape(lev))
        y = np.empty_like(u)
        _load().og_apply(self._h, lev, _dp(u), _dp(y))
        return y

    def residual(self, b, u, lev=0):
        b, u = _f64(b).reshape(self.shape(lev)), _f64(u).reshape(self.shape(lev))
        r = np.empty_like(u)
        _load().og_residual(self._h, lev, _dp(b), _dp(u), _dp(r))
        return r

    def dense(self, lev=0):
        N = self.ncol(lev) * self.nz
        M = np.empty((N, N))
        _load().og_assemble_dense(self._h, lev, _dp(M))
        return M

    # -- relaxation and transfers ------------------------------------------
    def smooth(self, b, u, nsweeps=1, rho=0.8, lev=0):
        b = _f64(b).reshape(self.shape(lev))
        u = _f64(u).reshape(self.shape(lev)).copy()
        _load().og_smooth(self._h, lev, _dp(b), _dp(u), nsweeps, rho)
        return u

    def rb_ssor(self, r, rho=1.0, lev=0):
        """z = M^{-1} r of the block red-black SSOR preconditioner."""
        r = _f64(r).reshape(self.shape(lev))
        z = np.empty_like(r)
        _load().og_rb_ssor(self._h, lev, _dp(r), _dp(z), rho)
        return z

    def colour(self, lev=0):
        """0 (red) or 1 (black) per column: parity of i + j."""
        n = self.level_n(lev)
        c = np.arange(self.ncol(lev))
        return ((c % n) + (c // n) % n) % 2

    def line_precond(self, r, lev=0):
        r = _f64(r).reshape(self.shape(lev))
        z = np.empty_like(r)
        _load().og_line_precond(self._h, lev, _dp(r), _dp(z))
        return z

    def restrict(self, r_f, lev_f=0):
        r_f = _f64(r_f).reshape(self.shape(lev_f))
        b_c = np.empty(self.shape(lev_f + 1))
        _load().og_restrict(self._h, lev_f, _dp(r_f), _dp(b_c))
        return b_c

    def prolong_add(self, u_c, u_f, lev_f=0, mode=0):
        u_c = _f64(u_c).reshape(self.shape(lev_f + 1))
        u_f = _f64(u_f).reshape(self.shape(lev_f)).copy()
        _load().og_prolong_add(self._h, lev_f, _dp(u_c), _dp(u_f), mode)
        return u_f

    # -- solvers ------------------------------------------------------------
    def vcycle(self, b, u, nu_pre=2, nu_post=2, nu_coarse=2, rho=0.8, rho_coarse=1.0,
               prolong_mode=0):
        b = _f64(b).reshape(self.shape())
        u = _f64(u).reshape(self.shape()).copy()
        _load().og_vcycle(self._h, _dp(b), _dp(u), nu_pre, nu_post, nu_coarse, rho,
                          rho_coarse, prolong_mode)
        return u

    def fmg(self, b, nu_pre=2, nu_post=2, nu_coarse=2, rho=0.8, rho_coarse=1.0, prolong_mode=0):
        """One full-multigrid cycle from zero; returns u."""
        b = _f64(b).reshape(self.shape())
        u = np.zeros_like(b)
        _load().og_fmg(self._h, _dp(b), _dp(u), nu_pre, nu_post, nu_coarse, rho, rho_coarse,
                       prolong_mode)
        return u

    def mg_solve(self, b, rtol=1e-5, maxit=50, nu_pre=2, nu_post=2, nu_coarse=2, rho=0.8,
                 rho_coarse=1.0, prolong_mode=0):
        b = _f64(b).reshape(self.shape())
        u = np.empty_like(b)
        hist = np.zeros(maxit + 1)
        it = _load().og_mg_solve(self._h, _dp(b), _dp(u), rtol, maxit, nu_pre, nu_post,
                                 nu_coarse, rho, rho_coarse, prolong_mode, _dp(hist))
        return u, it, hist[: it + 1]

    def pcg_solve(self, b, rtol=1e-5, maxit=500):
        b = _f64(b).reshape(self.shape())
        u = np.empty_like(b)
        hist = np.zeros(maxit + 1)
        it = _load().og_pcg_solve(self._h, _dp(b), _dp(u), rtol, maxit, _dp(hist))
        return u, it, hist[: it + 1]
