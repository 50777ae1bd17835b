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


def test_struct_layouts_match_header(lib, tmp_path):
    """The ctypes mirrors have the sizes and field offsets the C compiler gives the
    structs of include/ferrox.h (a small C program built against the header)."""
    import shutil
    import subprocess
    from paper_2210_15668_gb300 import ferrox
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"ferrox_layer": ferrox.Layer, "ferrox_geometry": ferrox.Geometry,
               "ferrox_numerics": ferrox.Numerics, "ferrox_charge_t": ferrox.Charge,
               "ferrox_stats": ferrox.Stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ferrox.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


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
