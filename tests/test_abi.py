"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2601_18417_gb300 import build, hofv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(hofv_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_api():
    names = declared_symbols()
    for must in ("hofv_create", "hofv_residual", "hofv_jvp", "hofv_precondition",
                 "hofv_newton_solve", "hofv_set_mesh", "hofv_set_material",
                 "hofv_build_stencils"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header():
    assert set(hofv.SIGNATURES) >= set(declared_symbols())


def test_version_string():
    lib = hofv.load()
    assert lib.hofv_version().startswith(b"hofv")
