"""The C ABI library loads and exports every symbol that include/pspc.h
declares (no GPU needed: nothing is called that computes)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(pspc_\w+)\s*\(", txt, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2212_00977_gb300 import build_lib

    path = build_lib.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"pspc_build", "pspc_query", "pspc_free", "pspc_export", "pspc_stats",
            "pspc_level_stats", "pspc_strerror"} <= set(names)
    for nm in names:
        assert hasattr(lib, nm), nm


def test_binding_signatures_cover_header(lib):
    import paper_2212_00977_gb300 as pspc

    assert set(declared_functions()) == set(pspc._SIGS)


def test_strerror_and_null_arguments_need_no_gpu(lib):
    import paper_2212_00977_gb300 as pspc

    L = pspc.load()
    assert L.pspc_strerror(0) == b"ok"
    assert b"invalid" in L.pspc_strerror(1)
    # NULL output handle / NULL index are rejected before any CUDA call
    assert L.pspc_build(None, None, None, None, None) == pspc.PSPC_E_INVAL
    assert L.pspc_query(None, None, 0, None, None, None, None) == pspc.PSPC_E_INVAL
    assert L.pspc_stats(None, None) == pspc.PSPC_E_INVAL
    L.pspc_free(None)


def test_product_path_has_no_oracle_or_cpu_fallback():
    """The package never imports the oracle, and loading fails loudly when
    the CUDA library is missing."""
    pkg = os.path.join(ROOT, "paper_2212_00977_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "pspc_oracle" not in txt, f
    import paper_2212_00977_gb300 as pspc

    with pytest.raises(RuntimeError):
        pspc.load("/nonexistent/libpspc.so")
