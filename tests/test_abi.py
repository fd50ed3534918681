"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point that include/*.h declares.  No compute calls."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(ms_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("ms_init", "ms_step", "ms_moments", "ms_truth_step"):
        assert core in names


def test_library_exports_every_declared_symbol():
    from paper_2303_07819_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_match_header():
    from paper_2303_07819_gb300 import msdem
    assert set(msdem.SYMBOLS) <= set(declared_symbols())


def test_oracle_is_not_imported_by_the_product_package():
    pkg = os.path.join(ROOT, "paper_2303_07819_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(f).read()
            assert "oracle" not in re.findall(r"^\s*(?:from|import)\s+(\w+)", src, flags=re.M), f
            assert "ms_oracle" not in src, f
