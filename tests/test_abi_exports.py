"""The C-ABI library builds, loads and exports every symbol that
include/matexpre.h declares (no compute calls: this runs without a GPU)."""
import ctypes as ct
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mxp_\w+)\s*\(", src))
    return names


def test_header_declares_the_core_entry_points():
    names = _declared()
    for required in ["mxp_create", "mxp_set_params", "mxp_apply_operator", "mxp_apply_matexpre",
                     "mxp_solve", "mxp_solve_batch", "mxp_destroy", "mxp_status_string",
                     "mxp_last_error", "mxp_apply_phi", "mxp_create_slab", "mxp_horner_step",
                     "mxp_vec_mdot", "mxp_vec_combine", "mxp_apply_phi_noalloc"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2506_03617_gb300 import build
    path = build.build()
    lib = ct.CDLL(path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2506_03617_gb300 import native
    assert _declared() <= set(native.SIGNATURES)


def test_status_strings_without_gpu():
    from paper_2506_03617_gb300 import native
    lib = native.load()
    assert lib.mxp_status_string(0) == b"ok"
    assert lib.mxp_status_string(4) == b"not converged"


def test_create_rejects_bad_input_before_touching_a_device():
    import numpy as np
    from paper_2506_03617_gb300 import native
    lib = native.load()
    g = native.Grid()
    g.dim = 4
    g.npml = 0
    g.h = 0.1
    out = ct.c_void_p()
    c = np.ones(8)
    s = lib.mxp_create(ct.byref(g), c.ctypes.data_as(ct.POINTER(ct.c_double)), 0, None,
                       ct.byref(out))
    assert s == 1 and b"dim" in lib.mxp_last_error()
    g.dim = 2
    g.n_interior[0] = 2
    g.n_interior[1] = 2
    c = np.array([1.0, 1.0, -1.0, 1.0])
    s = lib.mxp_create(ct.byref(g), c.ctypes.data_as(ct.POINTER(ct.c_double)), 0, None,
                       ct.byref(out))
    assert s == 1 and b"wave speed" in lib.mxp_last_error()
