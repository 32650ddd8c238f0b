"""The C-ABI library builds, loads and exports every symbol include/cc3.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    import glob
    txt = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cc3_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_2007_01088_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert "cc3_omega_triples" in names and "cc3_serve_start" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2007_01088_gb300 as g
    assert sorted(g.EXPORTED) == declared_symbols()


def test_strerror_and_argument_errors():
    import paper_2007_01088_gb300 as g
    assert g.cc3_strerror(0) == "ok"
    assert "timed out" in g.cc3_strerror(-4)
    ctx = ctypes.c_void_p()
    # invalid sizes are rejected before any device work
    assert g.lib.cc3_ctx_create(ctypes.byref(ctx), 0, 5, *([None] * 8), 0, 0, None) == -1
    assert g.lib.cc3_ctx_create(ctypes.byref(ctx), 3, 5, *([None] * 8), 0, 0, None) == -1
    assert g.lib.cc3_omega_triples(None, 0, None, None, None, None) == -1
