"""Thin ctypes binding of libellsolve.so (the C ABI of include/ellsolve.h).

Only argument marshalling happens here: every step of the solve runs in the
library's CUDA kernels.  Importing this module fails loudly if the library has
not been built (run __graft_entry__.build() or paper_1307_2036_gb300/build.py);
there is no CPU fallback.

Vectors are passed as device pointers; the helpers accept torch CUDA tensors
(float64 unless a level call asks for fp32) of shape (nz, P, n, n) or flat.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libellsolve.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: the ellsolve CUDA library has not been built "
        "(python -c 'import __graft_entry__ as g; g.build()')")

_lib = C.CDLL(LIB_PATH)

OK, NOT_CONVERGED, PENDING = 0, 1, 2
ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_NONFINITE, ERR_CAPACITY = -1, -2, -3, -4, -5
_STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "PENDING", -1: "ERR_ARG", -2: "ERR_CUDA",
           -3: "ERR_NOMEM", -4: "ERR_NONFINITE", -5: "ERR_CAPACITY"}


class ellsolve_grid(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("nz", C.c_int), ("box_side", C.c_double),
                ("mapping", C.c_int)]


class ellsolve_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("solver", C.c_int), ("nu_pre", C.c_int),
                ("nu_post", C.c_int), ("nu_coarse", C.c_int), ("damping", C.c_double),
                ("coarsest_min", C.c_int), ("max_levels", C.c_int), ("prolong", C.c_int),
                ("inner_cycles", C.c_int), ("use_graph", C.c_int), ("smoother", C.c_int),
                ("precond", C.c_int), ("fmg", C.c_int), ("refine", C.c_int),
                ("line_part", C.c_int)]


class ellsolve_result(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("seconds", C.c_double),
                ("rel_error_est", C.c_double)]


_vp, _i, _d, _st = C.c_void_p, C.c_int, C.c_double, C.c_int
_SIGS = {
    "ellsolve_default_opts": (None, [C.POINTER(ellsolve_opts)]),
    "ellsolve_create": (_st, [C.POINTER(ellsolve_grid), _d, _d, C.POINTER(C.c_double),
                              C.POINTER(ellsolve_opts), _vp, C.POINTER(_vp)]),
    "ellsolve_create_profiles": (_st, [C.POINTER(ellsolve_grid), _d, _d, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double),
                                       C.POINTER(ellsolve_opts), _vp, C.POINTER(_vp)]),
    "ellsolve_destroy": (None, [_vp]),
    "ellsolve_size": (C.c_size_t, [_vp]),
    "ellsolve_num_levels": (_i, [_vp]),
    "ellsolve_apply": (_st, [_vp, _vp, _vp]),
    "ellsolve_vcycle": (_st, [_vp, _vp, _vp]),
    "ellsolve_solve": (_st, [_vp, _vp, _vp, _d, _i, C.POINTER(ellsolve_result)]),
    "ellsolve_solve_batch": (_st, [C.POINTER(_vp), _i, C.POINTER(_vp), C.POINTER(_vp), _d, _i,
                                   C.POINTER(ellsolve_result)]),
    "ellsolve_level_shape": (_st, [_vp, _i, C.POINTER(_i), C.POINTER(C.c_size_t)]),
    "ellsolve_level_apply": (_st, [_vp, _i, _i, _vp, _vp]),
    "ellsolve_level_residual": (_st, [_vp, _i, _i, _vp, _vp, _vp]),
    "ellsolve_level_smooth": (_st, [_vp, _i, _i, _vp, _vp, _i, _d]),
    "ellsolve_level_restrict_residual": (_st, [_vp, _i, _i, _vp, _vp, _vp]),
    "ellsolve_level_prolong_add": (_st, [_vp, _i, _i, _vp, _vp]),
    "ellsolve_level_smooth_noalloc": (_st, [_vp, _i, _i, _vp, _vp, _i, _d]),
    "ellsolve_profile_enable": (_st, [_vp, _i]),
    "ellsolve_profile_read": (_st, [_vp, C.POINTER(_d), C.POINTER(_i), C.POINTER(_d)]),
    "ellsolve_launch_count": (C.c_uint64, [_vp]),
    "ellsolve_autotune": (_st, [_vp, C.POINTER(_i), C.POINTER(_d)]),
    "ellsolve_set_tuning": (_st, [_vp, _i, _i]),
    "ellsolve_selftest": (_st, [C.c_uint64, C.POINTER(C.c_uint64)]),
    "ellsolve_get_tuning": (_st, [_vp, C.POINTER(_i), C.POINTER(_i)]),
    "ellsolve_set_level_tuning": (_st, [_vp, _i, _i, _i, _i, _i, _i, _i]),
    "ellsolve_get_level_tuning": (_st, [_vp, _i] + [C.POINTER(_i)] * 6),
    "ellsolve_server_create": (_st, [C.c_size_t, _i, _vp, C.POINTER(_vp)]),
    "ellsolve_submit": (_st, [_vp, C.POINTER(ellsolve_grid), _d, _d, C.POINTER(C.c_double), _vp,
                              _vp, _d, _i, C.POINTER(C.c_uint64)]),
    "ellsolve_poll": (_st, [_vp, C.c_uint64, _i, C.POINTER(ellsolve_result)]),
    "ellsolve_server_destroy": (None, [_vp]),
    "ellsolve_last_error": (C.c_char_p, []),
}
EXPORTS = tuple(_SIGS)
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class EllsolveError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.ellsolve_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status, where="ellsolve"):
    if status < 0:
        raise EllsolveError(status, where)
    return status


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def default_opts(**kw):
    o = ellsolve_opts()
    _lib.ellsolve_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


class Solver:
    """One problem: grid, omega^2, lambda^2, radial levels and solver options."""

    def __init__(self, kind, n, nz, r_levels, omega2, lambda2, mapping=0, box_side=None,
                 stream=None, p_cell=None, q_face=None, **opts):
        import math
        g = ellsolve_grid(kind=kind, n=n, nz=nz,
                          box_side=2 * math.pi if box_side is None else box_side, mapping=mapping)
        o = default_opts(**opts)
        r = (C.c_double * (nz + 1))(*[float(v) for v in r_levels])
        self.stream = _current_stream() if stream is None else stream
        h = C.c_void_p()
        pc = None if p_cell is None else (C.c_double * nz)(*[float(v) for v in p_cell])
        qf = None if q_face is None else (C.c_double * (nz + 1))(*[float(v) for v in q_face])
        check(_lib.ellsolve_create_profiles(C.byref(g), float(omega2), float(lambda2), r, pc, qf,
                                            C.byref(o), C.c_void_p(self.stream), C.byref(h)),
              "ellsolve_create")
        self.h = h
        self.kind, self.n, self.nz, self.P = kind, n, nz, 1 if kind == 0 else 6
        self.opts = o
        self.N = _lib.ellsolve_size(h)
        self.nlevels = _lib.ellsolve_num_levels(h)

    def close(self):
        if getattr(self, "h", None):
            _lib.ellsolve_destroy(self.h)
            self.h = None

    __del__ = close

    def shape(self, level=0):
        n = C.c_int()
        nc = C.c_size_t()
        check(_lib.ellsolve_level_shape(self.h, level, C.byref(n), C.byref(nc)), "level_shape")
        return (self.nz, self.P, n.value, n.value)

    def apply(self, x, y):
        return check(_lib.ellsolve_apply(self.h, _ptr(x), _ptr(y)), "ellsolve_apply")

    def vcycle(self, f, u):
        return check(_lib.ellsolve_vcycle(self.h, _ptr(f), _ptr(u)), "ellsolve_vcycle")

    def solve(self, f, x, rtol=1e-5, maxit=50):
        res = ellsolve_result()
        st = check(_lib.ellsolve_solve(self.h, _ptr(f), _ptr(x), float(rtol), int(maxit),
                                       C.byref(res)), "ellsolve_solve")
        return st, res

    # kernel-level access (volume-integrated b)
    def level_apply(self, level, x, y, fp32=False):
        return check(_lib.ellsolve_level_apply(self.h, level, int(fp32), _ptr(x), _ptr(y)), "level_apply")

    def level_residual(self, level, b, u, r, fp32=False):
        return check(_lib.ellsolve_level_residual(self.h, level, int(fp32), _ptr(b), _ptr(u), _ptr(r)),
                     "level_residual")

    def level_smooth(self, level, b, u, nsweeps=1, rho=0.8, fp32=False):
        return check(_lib.ellsolve_level_smooth(self.h, level, int(fp32), _ptr(b), _ptr(u),
                                                int(nsweeps), float(rho)), "level_smooth")

    def level_restrict_residual(self, level, b, u, b_c, fp32=False):
        return check(_lib.ellsolve_level_restrict_residual(self.h, level, int(fp32), _ptr(b), _ptr(u),
                                                           _ptr(b_c)), "level_restrict_residual")

    def level_prolong_add(self, level, u_c, u, fp32=False):
        return check(_lib.ellsolve_level_prolong_add(self.h, level, int(fp32), _ptr(u_c), _ptr(u)),
                     "level_prolong_add")

    def profile(self, enable=True):
        check(_lib.ellsolve_profile_enable(self.h, int(enable)), "profile_enable")

    def profile_read(self):
        ms, n, b = C.c_double(), C.c_int(), C.c_double()
        check(_lib.ellsolve_profile_read(self.h, C.byref(ms), C.byref(n), C.byref(b)), "profile_read")
        return ms.value, n.value, b.value

    def launch_count(self):
        return int(_lib.ellsolve_launch_count(self.h))

    def autotune(self):
        """Pick the smoother's CTAs per SM by timing; returns (ctas, ms per sweep)."""
        c, ms = C.c_int(), C.c_double()
        check(_lib.ellsolve_autotune(self.h, C.byref(c), C.byref(ms)), "ellsolve_autotune")
        return c.value, ms.value

    def set_tuning(self, ctas_per_sm, ring):
        check(_lib.ellsolve_set_tuning(self.h, int(ctas_per_sm), int(ring)), "set_tuning")

    def tuning(self):
        """(resident CTAs per SM, ring depth) of the FP32 line smoother."""
        c, r = C.c_int(), C.c_int()
        check(_lib.ellsolve_get_tuning(self.h, C.byref(c), C.byref(r)), "get_tuning")
        return c.value, r.value

    def set_level_tuning(self, level, ctas_per_sm, ring, tmem=0, staged=0, restrict_chunk=608,
                         prolong_chunk=608):
        check(_lib.ellsolve_set_level_tuning(self.h, int(level), int(ctas_per_sm), int(ring),
                                             int(tmem), int(staged), int(restrict_chunk),
                                             int(prolong_chunk)),
              "set_level_tuning")

    def level_tuning(self, level):
        """(ctas per SM, ring, tmem, staged, restrict chunk, prolong chunk) of one level."""
        v = [C.c_int() for _ in range(6)]
        check(_lib.ellsolve_get_level_tuning(self.h, int(level), *[C.byref(x) for x in v]),
              "get_level_tuning")
        return tuple(x.value for x in v)


def selftest(samples=1 << 24):
    """Device self-check of the library's integer-arithmetic conversions;
    returns the number of mismatches (raises if there are any)."""
    bad = C.c_uint64()
    check(_lib.ellsolve_selftest(int(samples), C.byref(bad)), "ellsolve_selftest")
    return bad.value


def solve_batch(solvers, rhs, xs, rtol=1e-8, maxit=50):
    """One batched solve over several Solver objects (precision 1, MG)."""
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
    rp = (C.c_void_p * n)(*[_ptr(t) for t in rhs])
    xp = (C.c_void_p * n)(*[_ptr(t) for t in xs])
    res = (ellsolve_result * n)()
    st = check(_lib.ellsolve_solve_batch(hs, n, rp, xp, float(rtol), int(maxit), res), "solve_batch")
    return st, list(res)


class Server:
    """Continuous-batching request server (ellsolve_server_*).  The caller keeps
    each request's rhs and x tensors alive and leaves them untouched until its
    poll returns a final status; rhs must be fully written before submit."""

    def __init__(self, hbm_budget_bytes, max_slots, stream=None):
        self.stream = _current_stream() if stream is None else stream
        h = C.c_void_p()
        check(_lib.ellsolve_server_create(C.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                          C.c_void_p(self.stream), C.byref(h)),
              "ellsolve_server_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.ellsolve_server_destroy(self.h)
            self.h = None

    __del__ = close

    def submit(self, kind, n, nz, r_levels, omega2, lambda2, f, x, rtol=1e-5, maxit=50,
               mapping=0, box_side=None):
        import math
        g = ellsolve_grid(kind=kind, n=n, nz=nz,
                          box_side=2 * math.pi if box_side is None else box_side, mapping=mapping)
        r = (C.c_double * (nz + 1))(*[float(v) for v in r_levels])
        t = C.c_uint64()
        check(_lib.ellsolve_submit(self.h, C.byref(g), float(omega2), float(lambda2), r, _ptr(f),
                                   _ptr(x), float(rtol), int(maxit), C.byref(t)), "ellsolve_submit")
        return t.value

    def poll(self, ticket, timeout_us=-1):
        """Returns (status, result); status PENDING if not finished in time."""
        res = ellsolve_result()
        st = _lib.ellsolve_poll(self.h, C.c_uint64(ticket), int(timeout_us), C.byref(res))
        if st < 0 and st != ERR_NONFINITE:
            raise EllsolveError(st, "ellsolve_poll")
        return st, res
