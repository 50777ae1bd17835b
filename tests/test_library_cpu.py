"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point that include/ferrox.h declares (no compute calls)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"\b(ferrox_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2210_15668_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ferrox_init_geometry", "ferrox_set_bias", "ferrox_step", "ferrox_solve_poisson",
              "ferrox_charge"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(declared_symbols()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2210_15668_gb300 import ferrox
    assert declared_symbols() <= set(ferrox.EXPORTS) | {"ferrox_status"}


def test_struct_layouts_match_header(lib):
    """The ctypes mirrors have the sizes the C compiler gives the structs."""
    from paper_2210_15668_gb300 import ferrox
    assert ctypes.sizeof(ferrox.Layer) == 8 + 14 * 8
    assert ctypes.sizeof(ferrox.Numerics) == 8 + 4 + 4 + 8 + 5 * 4 + 4 + 4 + 4
    assert ctypes.sizeof(ferrox.Stats) == 4 * 8 + 8 + 8 + 8 + 8 + 8


def test_init_rejects_bad_arguments_without_gpu(lib):
    """Argument validation runs before any CUDA call."""
    from paper_2210_15668_gb300 import ferrox
    L = ferrox.make_layers([dict(kind=1, ncells=4, eps_r=3.9)])
    g = ferrox.Geometry(8, 8, 0.5e-9, 1, L, 0, 0.0, 1)
    n = ferrox.make_numerics(4e-13)
    ctx = ctypes.c_void_p()
    lib.ferrox_last_error.restype = ctypes.c_char_p
    rc = lib.ferrox_init_geometry(ctypes.byref(ctx), ctypes.byref(g), ctypes.byref(n),
                                  ctypes.c_void_p(4096), ctypes.c_void_p(8192), None)
    assert rc == ferrox.FERROX_EINVAL
    assert b"ferroelectric" in lib.ferrox_last_error(None)
