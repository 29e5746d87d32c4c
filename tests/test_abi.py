"""The C ABI library loads without a GPU and exports every function declared in include/*.h;
the Python binding declares a signature for each one (no compute calls here)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fft_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fft_table_build", "fft_geom_create", "fft_J_apply", "fft_JT_apply", "fft_cg_solve",
                     "fft_psf_batch", "fft_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_1908_03302_gb300 import _lib
    L = _lib.load()
    for name in declared_functions():
        assert hasattr(L, name), name
        assert name in _lib.SIGNATURES, name
    assert L.fft_last_error() == b""


def test_oracle_is_not_imported_by_the_product():
    pkg = os.path.join(ROOT, "paper_1908_03302_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "fft_oracle" not in text, path


def test_fresnel_width_printed_value():
    # Sec. IV: c0 = 1479.7 m/s, L_max = 0.19 m, fc = 3.2 MHz give a 9.4 mm Fresnel width.
    from paper_1908_03302_gb300 import fresnel_width
    assert round(fresnel_width(1479.7, 0.19, 3.2e6) * 1e3, 1) == 9.4
