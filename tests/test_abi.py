"""The C-ABI library loads and exports every function include/*.h declares;
host-side argument validation answers without touching a GPU."""
import ctypes as C
import glob
import os
import re

import pytest

from conftest import ROOT


def _lib():
    from paper_1804_00462_gb300 import _build
    if not os.path.exists(_build.LIB):
        _build.build()
    return C.CDLL(_build.LIB)


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\**\s+(sorsvd_\w+)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = _declared()
    assert {"sorsvd_run", "sorsvd_workspace_size", "sorsvd_gaussian", "sorsvd_get_status"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings_and_workspace_validation():
    lib = _lib()
    lib.sorsvd_status_string.restype = C.c_char_p
    assert lib.sorsvd_status_string(0) == b"ok"
    assert b"workspace" in lib.sorsvd_status_string(7)
    ws = lib.sorsvd_workspace_size
    ws.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint]
    ws.restype = C.c_size_t
    assert ws(1000, 1000, 20, 5, 0, 0) > 0
    assert ws(1000, 1000, 0, 5, 0, 0) == 0          # k < 1
    assert ws(1000, 1000, 20, -1, 0, 0) == 0        # p < 0
    assert ws(10, 1000, 20, 5, 0, 0) == 0           # l > min(m, n)
    assert ws(1000, 1000, 20, 5, 9, 0) == 0         # unknown dtype
    assert ws(5000, 5000, 200, 30, 0, 0) == 0       # l > SORSVD_MAX_L_F64
    assert ws(5000, 5000, 300, 20, 1, 0) > 0        # l = 320 fits fp32 factors
    assert ws(5000, 5000, 300, 21, 1, 0) == 0


def test_run_rejects_bad_arguments_before_any_device_work():
    lib = _lib()
    f = lib.sorsvd_run
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                  C.c_uint, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t,
                  C.c_void_p]
    fake = 0x1000
    ok = dict(A=fake, m=100, n=80, lda=100, k=5, p=5, q=1, seed=0, dt=1, fl=0, U=fake, ldu=100, S=fake,
              V=fake, ldv=80, ws=None, wsb=0, st=None)

    def call(**kw):
        a = dict(ok, **kw)
        return f(a["A"], a["m"], a["n"], a["lda"], a["k"], a["p"], a["q"], a["seed"], a["dt"], a["fl"],
                 a["U"], a["ldu"], a["S"], a["V"], a["ldv"], a["ws"], a["wsb"], a["st"])
    assert call(A=None) == 1
    assert call(lda=99) == 1
    assert call(ldu=50) == 1
    assert call(ldv=79) == 1
    assert call(k=0) == 1
    assert call(p=-1) == 1
    assert call(q=-1) == 1
    assert call(k=80, p=1) == 1                     # l > min(m, n)
    assert call(fl=0x80) == 1                       # unknown flag
    assert call(dt=7) == 2
    assert call() == 7                              # no workspace
    assert call(ws=0x1010, wsb=1 << 30) == 7        # misaligned workspace
    assert call(ws=0x1000, wsb=16) == 7             # too small
