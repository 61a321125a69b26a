"""CPU checks of the C-ABI library: it builds, loads, and exports every
function include/dem.h declares; host-only entry points behave.  No GPU work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(dem_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    import shutil
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2311_11322_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_exported(lib):
    names = declared_functions()
    assert "dem_step" in names and "dem_add_aggregates" in names and len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2311_11322_gb300 import dem
    import inspect
    src = inspect.getsource(dem.load)
    for n in declared_functions():
        assert f'"{n}"' in src, n


def test_footprint_is_host_only_and_monotone(lib):
    f = lib.dem_footprint_bytes
    f.restype = C.c_size_t
    f.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32]
    a = f(1000, 250, 16, 1)
    b = f(100000, 25000, 16, 1)
    c = f(100000, 25000, 16, 0)
    assert 0 < a < b < c
    assert f(-1, 0, 16, 1) == 0


def test_last_error_null_world(lib):
    g = lib.dem_last_error
    g.restype = C.c_char_p
    g.argtypes = [C.c_void_p]
    assert g(None) == b"NULL world"


def test_params_struct_layout():
    """The ctypes mirror of dem_params has the C layout (offsets of the int
    fields and of the trailing arrays)."""
    from paper_2311_11322_gb300 import dem
    P = dem.dem_params
    assert P.precision.offset == 88 and P.max_contacts.offset == 92
    assert P.cell_size.offset == 96 and P.spin_inc.offset == 160
    assert P.rot_tol.offset == 184 and C.sizeof(P) == 192
