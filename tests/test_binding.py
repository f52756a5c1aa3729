"""The Python binding against the C header, without a GPU: the ctypes
structures list the header's struct fields in the same order with the same
widths, and bad argument types are rejected before the library is called."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CTYPE = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float}


def header_struct(name):
    """(field, type) pairs of `typedef struct { ... } name;` in pspc.h."""
    txt = open(os.path.join(ROOT, "include", "pspc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + re.escape(name) + r"\s*;", txt)
    assert m, name
    fields = []
    for line in m.group(1).split(";"):
        line = line.strip()
        if not line:
            continue
        typ, _, field = line.rpartition(" ")
        fields.append((field.strip("*"), typ.strip()))
    return fields


@pytest.mark.parametrize("cname,pyname", [("pspc_opts", "Opts"), ("pspc_stats_t", "Stats"),
                                          ("pspc_level_stat_t", "LevelStat")])
def test_structs_match_header(cname, pyname):
    import paper_2212_00977_gb300 as pspc

    want = header_struct(cname)
    got = getattr(pspc, pyname)._fields_
    assert [f for f, _ in got] == [f for f, _ in want]
    for (f, ct), (_, ht) in zip(got, want):
        assert ct == CTYPE[ht], (f, ht)


def test_bad_dtypes_are_rejected_before_the_call():
    import paper_2212_00977_gb300 as pspc
    from paper_2212_00977_gb300 import build_lib

    build_lib.build()
    rp = np.array([0, 1, 2], np.int64)
    col = np.array([1, 0], np.int32)
    rank = np.array([0, 1], np.int32)
    with pytest.raises(TypeError):
        pspc.Index.build(2, rp.astype(np.int32), col, rank)
    with pytest.raises(TypeError):
        pspc.Index.build(2, rp, col.astype(np.int64), rank)
    with pytest.raises(TypeError):
        pspc.Index.build(2, rp, col, rank.astype(np.int64))
    ix = pspc.Index(0, 2)  # a null handle: only the argument checks run
    with pytest.raises(TypeError):
        ix.query(np.zeros((1, 2), np.int64))
