"""The C-ABI library loads and exports every function include/ellsolve.h
declares (CPU only: nothing is called that would need a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ellsolve.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(ellsolve_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ellsolve_create", "ellsolve_apply", "ellsolve_vcycle", "ellsolve_solve",
                     "ellsolve_submit", "ellsolve_poll", "ellsolve_destroy",
                     "ellsolve_server_create", "ellsolve_server_destroy", "ellsolve_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1307_2036_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding wraps exactly these names
    from paper_1307_2036_gb300 import ellsolve
    assert set(ellsolve.EXPORTS) == set(declared_functions())


def test_default_opts_without_gpu():
    from paper_1307_2036_gb300 import ellsolve
    o = ellsolve.default_opts()
    assert (o.nu_pre, o.nu_post, o.nu_coarse, o.coarsest_min) == (2, 2, 2, 4)
    assert abs(o.damping - 0.8) < 1e-15


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    from paper_1307_2036_gb300 import ellsolve
    g = ellsolve.ellsolve_grid(kind=0, n=8, nz=4, box_side=6.28, mapping=0)
    r = (ctypes.c_double * 5)(1.0, 1.01, 1.005, 1.02, 1.03)  # not increasing
    h = ctypes.c_void_p()
    st = ellsolve.ellsolve_create(ctypes.byref(g), 0.01, 1.0, r, None, None, ctypes.byref(h))
    assert st == ellsolve.ERR_ARG and not h.value
    assert b"increasing" in ellsolve.ellsolve_last_error()


def test_binding_structs_match_the_header():
    """The ctypes mirrors of ellsolve_grid, ellsolve_opts and ellsolve_result
    list the header's fields in the header's order."""
    import re
    from paper_1307_2036_gb300 import ellsolve
    text = open(os.path.join(ROOT, "include", "ellsolve.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    structs = {m.group(2): m.group(1)
               for m in re.finditer(r"typedef struct \{([^{}]*)\}\s*(\w+);", text)}
    for name in ("ellsolve_grid", "ellsolve_opts", "ellsolve_result"):
        fields = re.findall(r"\b(?:int|double)\s+(\w+);", structs[name])
        assert [f for f, _ in getattr(ellsolve, name)._fields_] == fields, name
