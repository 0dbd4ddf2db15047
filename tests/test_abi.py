"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/vof.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vof.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vof_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vof_reconstruct", "vof_flux_polyhedra", "vof_correct_flux", "vof_phase_flux",
                     "vof_advect", "vof_create", "vof_destroy", "vof_status", "vof_error_string"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1305_3417_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1305_3417_gb300 import vof
    assert set(vof.EXPORTS) <= set(declared_functions())


def test_error_strings_without_gpu():
    from paper_1305_3417_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.vof_error_string.restype = ctypes.c_char_p
    assert lib.vof_error_string(0) == b"ok"
    assert b"mesh" in lib.vof_error_string(-3)


def test_create_rejects_bad_arguments_without_gpu():
    """Argument checks run on the host before any device work."""
    from paper_1305_3417_gb300 import build, vof
    build.build()
    L = vof.lib()
    h = ctypes.c_void_p()
    assert L.vof_create(None, None, ctypes.byref(h)) == -1
    m = vof._Mesh(0, 0, 0, 0, None, None, None, None, None, None, None, None)
    assert L.vof_create(ctypes.byref(m), None, ctypes.byref(h)) == -1


def test_binding_fails_loudly_when_library_missing(monkeypatch):
    from paper_1305_3417_gb300 import vof
    monkeypatch.setattr(vof, "_lib", None)
    monkeypatch.setattr(vof, "LIB_PATH", "/nonexistent/libvof.so")
    with pytest.raises(vof.VofError):
        vof.lib()


def test_batch_and_network_reject_bad_arguments_without_gpu():
    """The batch and network entry points check their arguments on the host
    before any device work: bad case offsets, a batch size below one tile."""
    import numpy as np
    from paper_1305_3417_gb300 import build, vof
    build.build()
    L = vof.lib()
    h = ctypes.c_void_p()
    m = vof._Mesh(0, 0, 0, 8, None, None, None, None, None, None, None, None)
    o = vof._Options(1e-9, 1, 1, 0)
    for off in ([0, 4, 4, 8], [1, 8], [0, 7], [0, 9, 8]):   # empty case, bad first/last, decreasing
        cp = np.asarray(off, np.int32)
        assert L.vof_batch_create(ctypes.byref(m), cp.ctypes.data, cp.size - 1, ctypes.byref(o),
                                  ctypes.byref(h)) == -1, off
    assert L.vof_batch_create(ctypes.byref(m), None, 1, ctypes.byref(o), ctypes.byref(h)) == -1
    p = np.zeros(vof.MLP_NPARAM, np.float32)
    assert L.vof_mlp_create(8, p.ctypes.data, 0, ctypes.byref(h)) == -1          # below 16 samples
    assert L.vof_mlp_create(64, None, 0, ctypes.byref(h)) == -1
    assert L.vof_batch_advect(None, None, None, None, None, None, None) == -1
    assert L.vof_set_guess(None, None) == -1
