"""The C-ABI library loads and exports every symbol include/mf.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree():
    from paper_2608_27423_b300 import _lib
    assert declared_symbols() == sorted(_lib.EXPORTS)


def test_library_exports_all_symbols():
    from paper_2608_27423_b300 import build, _lib
    build.build()
    lib = _lib.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_argument_errors_without_gpu():
    """Host-side argument validation rejects bad meshes before touching a device."""
    import ctypes as C
    import numpy as np
    from paper_2608_27423_b300 import _lib
    lib = _lib.load()
    out = C.c_void_p()
    x0 = np.zeros((4, 2))
    z = np.zeros(4, np.uint8)
    cells = np.array([[0, 1, 2, 7]], np.int32)            # node id 7 out of range
    cs = np.zeros(1, np.uint8)
    ifc = np.zeros((1, 1), np.int32)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    st = lib.mf_mesh_from_arrays(2, 1, 4, p(x0), p(z), p(z), 1, p(cells), p(cs), 0.5, 1, 1, 1.0, 0.0, p(ifc), p(ifc),
                                 C.byref(out))
    assert st == _lib.MF_ERR_ARG
    st = lib.mf_mesh_from_arrays(4, 1, 4, p(x0), p(z), p(z), 1, p(cells), p(cs), 0.5, 1, 1, 1.0, 0.0, p(ifc), p(ifc),
                                 C.byref(out))
    assert st == _lib.MF_ERR_ARG
    o = _lib.MfSolverOpts()
    lib.mf_solver_defaults(C.byref(o))
    assert o.newton_rtol == 1e-8 and o.restart == 50
