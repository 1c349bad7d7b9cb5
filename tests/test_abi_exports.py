"""The C-ABI library loads and exports every function the headers declare
(CPU only: nothing is called)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ab_\w+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return names


def _lib_path():
    import __graft_entry__ as g
    mod = g._load_build_module()
    try:
        return mod.build()
    except RuntimeError as e:       # no nvcc on this machine
        pytest.skip(str(e))


def test_headers_declare_the_api():
    names = _declared()
    for n in ["ab_create", "ab_destroy", "ab_build", "ab_pair_sum", "ab_pair_sum_bwd",
              "ab_pair_list", "ab_kernel_matvec", "ab_kernel_matvec_bwd", "ab_bd_step",
              "ab_sync", "ab_status_string"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_headers():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_abi", os.path.join(ROOT, "paper_1704_08907_gb300", "_abi.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert set(mod.SIGNATURES) == _declared()


def test_status_strings_without_gpu():
    lib = ctypes.CDLL(_lib_path())
    lib.ab_status_string.restype = ctypes.c_char_p
    for s in range(9):
        assert lib.ab_status_string(s)
    assert lib.ab_status_string(99) == b"unknown status"


def _declared_arity():
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ab_\w+)\s*\(([^;{]*?)\)\s*;", txt, re.M | re.S):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_headers():
    """Every ctypes signature has exactly the parameters its declaration has
    (a missing or extra argument would pass garbage across the boundary)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_abi", os.path.join(ROOT, "paper_1704_08907_gb300", "_abi.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    arity = _declared_arity()
    assert set(arity) == _declared()
    bad = {n: (arity[n], len(mod.SIGNATURES[n][1])) for n in arity
           if arity[n] != len(mod.SIGNATURES[n][1])}
    assert not bad, bad
