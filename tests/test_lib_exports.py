"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/vie.h declares (no GPU needed: nothing is computed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("vie_", "hom_"))))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vie_setup", "vie_solve", "vie_farfield", "vie_farfield_dirs", "hom_transfer",
                     "vie_get_current", "vie_destroy", "vie_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(vielib):
    lib = ctypes.CDLL(vielib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    assert set(declared_functions()) <= set(vielib.EXPORTS) | {"vie_default_opts"}


def test_binding_loads_and_reports_errors_without_gpu(vielib):
    L = vielib.load()
    # pure host entry points work without a device
    o = vielib.default_opts()
    assert abs(o.tol - 1e-6) < 1e-18 and o.restart == 30
    code = L.hom_transfer(None, None, 1.2, None, 0, None, None, None)
    assert code == vielib.VIE_EINVAL
    assert b"bad arguments" in L.vie_last_error()


def test_options_struct_matches_the_header(vielib):
    """vie_default_opts writes exactly sizeof(vie_solve_opts) bytes: a buffer
    one struct long plus a fenced tail keeps its tail, and the binding's last
    field is set (a shorter or longer ctypes mirror would break one of the two)."""
    L = vielib.load()
    size = ctypes.sizeof(vielib._Opts)
    buf = (ctypes.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    L.vie_default_opts(ctypes.cast(buf, ctypes.POINTER(vielib._Opts)))
    assert all(b == 0xAB for b in buf[size:])
    o = vielib._Opts.from_buffer(buf)
    assert o.arnoldi == 1 and abs(o.inner_floor - 0.7) < 1e-15 and abs(o.reorth_eta - 0.1) < 1e-15
    import pytest
    with pytest.raises(TypeError):
        vielib.default_opts(no_such_option=1)
