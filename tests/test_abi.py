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


def test_run_host_sizes_and_rejects_bad_arguments_before_any_device_work():
    lib = _lib()
    ws = lib.sorsvd_workspace_size
    ws.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint]
    ws.restype = C.c_size_t
    host_io = 0x4
    for m, n, k, p, dt, esz in ((20000, 10000, 100, 10, 1, 4), (1000, 700, 20, 5, 3, 2), (300, 200, 10, 4, 0, 8)):
        base, host = ws(m, n, k, p, dt, 0), ws(m, n, k, p, dt, host_io)
        acc = 8 if dt == 0 else 4
        # the device copies of A, U, S, V come on top of the solve's workspace
        assert host >= base + m * n * esz + (m * k + k + n * k) * acc
        assert host % 256 == 0
    assert ws(10, 1000, 20, 5, 1, host_io) == 0     # l > min(m, n)
    f = lib.sorsvd_run_host
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
    assert call(S=None) == 1
    assert call(lda=99) == 1
    assert call(k=80, p=1) == 1
    assert call(fl=0x80) == 1
    assert call(dt=7) == 2
    assert call() == 7                              # no workspace
    assert call(fl=host_io) == 7                    # the flag is accepted; still no workspace
    # a workspace that fits sorsvd_run but not the device copies of A and the factors
    base = ws(100, 80, 5, 5, 1, 0)
    assert call(ws=0x100000, wsb=base) == 7
    assert call(ws=0x100010, wsb=1 << 30) == 7      # misaligned


def test_polar_inv_rejects_bad_arguments_before_any_device_work():
    lib = _lib()
    f = lib.sorsvd_polar_inv
    f.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    fake = 0x1000
    assert f(None, 10, fake, fake, fake, 1 << 20, None) == 1
    assert f(fake, 0, fake, fake, fake, 1 << 20, None) == 1
    assert f(fake, 321, fake, fake, fake, 1 << 30, None) == 8    # beyond SORSVD_MAX_L
    assert f(fake, 110, fake, fake, fake, 16, None) == 7         # scratch too small
    assert f(fake, 110, fake, fake, fake + 4, 1 << 20, None) == 7  # scratch misaligned


def test_rpca_rejects_bad_arguments_before_any_device_work():
    from paper_1804_00462_gb300 import native as nat
    lib = nat.lib
    fake = 0x1000
    prob = nat.RpcaProblem(fake, 1000, 100, 1000, fake, 1000, fake, 1000, 10.0, 0)
    arr = (nat.RpcaProblem * 1)(prob)
    it = (C.c_int * 1)()
    xi = (C.c_double * 1)()

    def call(arr=arr, batch=1, k=5, p=5, q=1, dt=nat.F32, fl=0, tol=1e-7, mi=50, rho=1.5, ws=None, wsb=0):
        return lib.sorsvd_rpca(arr, batch, k, p, q, dt, fl, tol, mi, rho, it, xi, None, ws, wsb, None)
    assert call(dt=nat.BF16) == 2
    assert call(dt=nat.F16) == 2
    assert call(fl=0x1) == 1
    assert call(batch=0) == 1
    assert call(tol=0.0) == 1
    assert call(mi=0) == 1
    assert call(rho=0.5) == 1
    assert call(q=-1) == 1
    assert call(k=0) == 1
    assert call(k=96, p=5) == 1                    # l = 101 > min(m, n)
    bad = (nat.RpcaProblem * 1)(nat.RpcaProblem(fake, 1000, 100, 999, fake, 1000, fake, 1000, 10.0, 0))
    assert call(arr=bad) == 1                      # ldx < m
    nul = (nat.RpcaProblem * 1)(nat.RpcaProblem(None, 1000, 100, 1000, fake, 1000, fake, 1000, 10.0, 0))
    assert call(arr=nul) == 1
    assert call() == 7                             # no workspace
    need = lib.sorsvd_rpca_workspace_size(arr, 1, 5, 5, nat.F32, 0)
    assert need > 2 * 1000 * 100 * 4
    assert call(ws=256, wsb=need - 1) == 7
    assert lib.sorsvd_rpca_workspace_size(arr, 1, 5, 5, nat.BF16, 0) == 0
    mixed = lib.sorsvd_rpca_workspace_size(arr, 1, 5, 5, nat.F32, nat.RPCA_FINISH_F64)
    assert mixed >= need + 1000 * 100 * 8          # + the binary64 copy of G
    assert call(fl=nat.RPCA_FINISH_F64, ws=256, wsb=mixed - 1) == 7


def test_batched_rejects_bad_arguments_before_any_device_work():
    from paper_1804_00462_gb300 import native as nat
    lib = nat.lib
    fake = 0x1000

    def prob(**kw):
        d = dict(A=fake, m=300, n=200, lda=300, k=10, p=8, q=1, seed=0, U=fake, ldu=300, S=fake, V=fake, ldv=200)
        d.update(kw)
        return nat.Problem(d["A"], d["m"], d["n"], d["lda"], d["k"], d["p"], d["q"], d["seed"], d["U"], d["ldu"],
                           d["S"], d["V"], d["ldv"])

    def arr(*ps):
        return (nat.Problem * len(ps))(*ps)
    good = arr(prob(), prob(m=50, n=400, lda=50, ldu=50, ldv=400, k=3, p=2, q=0))
    assert lib.sorsvd_batched_workspace_size(good, 2, nat.F32, 0) > 0
    assert lib.sorsvd_batched_workspace_size(good, 2, nat.F64, 0) > lib.sorsvd_batched_workspace_size(good, 2, nat.F32, 0)
    assert lib.sorsvd_batched_workspace_size(good, 0, nat.F32, 0) == 0
    assert lib.sorsvd_batched_workspace_size(good, 2, nat.BF16, 0) == 0
    assert lib.sorsvd_batched_workspace_size(good, 2, nat.F32, nat.FLAG_REFINE) == 0
    assert lib.sorsvd_batched_workspace_size(arr(prob(lda=299)), 1, nat.F32, 0) == 0
    assert lib.sorsvd_batched_workspace_size(arr(prob(k=195, p=10)), 1, nat.F32, 0) == 0   # l > min(m, n)
    h = C.c_void_p()

    def create(a, n, dt=nat.F32, fl=0, ws=None, wsb=0):
        return lib.sorsvd_batched_plan_create(C.byref(h), a, n, dt, fl, 0, ws, wsb, None)
    assert create(good, 2, dt=nat.F16) == 2
    assert create(good, 2, fl=0x80) == 1
    assert create(arr(prob(A=None)), 1) == 1
    assert create(arr(prob(m=2000, n=2000, lda=2000, ldu=2000, ldv=2000, k=150, p=20)), 1) == 8   # l > 160
    assert create(arr(prob(m=2000, n=2000, lda=2000, ldu=2000, ldv=2000, k=120, p=9)), 1, dt=nat.F64) == 8
    assert create(good, 2) == 7                      # no workspace
    assert h.value is None
    need = lib.sorsvd_batched_workspace_size(good, 2, nat.F32, 0)
    assert create(good, 2, ws=256, wsb=need - 1) == 7
    assert lib.sorsvd_batched_plan_launch(None, None) == 1
    lib.sorsvd_batched_plan_destroy(None)


def test_streamed_sizes_and_rejects_bad_arguments_before_any_device_work():
    lib = _lib()
    sz = lib.sorsvd_streamed_workspace_size
    sz.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int64]
    sz.restype = C.c_size_t
    ws = lib.sorsvd_workspace_size
    ws.argtypes = [C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint]
    ws.restype = C.c_size_t
    m, n, k, p = 200000, 4096, 100, 10
    for dt, esz in ((1, 4), (3, 2), (0, 8)):
        small, big = sz(m, n, k, p, dt, 8192), sz(m, n, k, p, dt, 65536)
        # two device blocks of rows of A (ld rounded to 16) on top of the sketches
        assert small > 0 and big > small and big - small >= 2 * (65536 - 8192) * n * esz
        assert small % 256 == 0 and big % 256 == 0
    # a block as large as A: no smaller than the in-core workspace without its copy of A^T
    assert sz(20000, 10000, 100, 10, 3, 20000) >= ws(20000, 10000, 100, 10, 3, 0)
    assert sz(m, n, 0, p, 1, 8192) == 0                # k < 1
    assert sz(m, n, k, p, 1, 0) == 0                   # no rows per block
    assert sz(100, 50, 45, 10, 1, 16) == 0             # l > min(m, n)
    assert sz(m, n, k, p, 9, 8192) == 0                # unknown dtype
    f = lib.sorsvd_run_streamed
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                  C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t,
                  C.c_void_p]
    fake = 0x1000
    ok = dict(A=fake, m=1000, n=800, lda=1000, k=20, p=5, q=1, seed=0, dt=1, br=256, U=fake, ldu=1000, S=fake,
              V=fake, ldv=800, ws=None, wsb=0, st=None)

    def call(**kw):
        a = dict(ok, **kw)
        return f(a["A"], a["m"], a["n"], a["lda"], a["k"], a["p"], a["q"], a["seed"], a["dt"], a["br"], a["U"],
                 a["ldu"], a["S"], a["V"], a["ldv"], a["ws"], a["wsb"], a["st"])
    assert call(A=None) == 1
    assert call(V=None) == 1
    assert call(lda=999) == 1
    assert call(ldv=799) == 1
    assert call(br=0) == 1
    assert call(k=800, p=1) == 1                       # l > min(m, n)
    assert call(k=400, p=0) == 8                       # l beyond the fp32 limit
    assert call(dt=7) == 2
    assert call() == 7                                 # no workspace
    need = sz(1000, 800, 20, 5, 1, 256)
    assert call(ws=0x100000, wsb=need - 256) == 7      # too small
    assert call(ws=0x100010, wsb=need) == 7            # misaligned


def test_products_size_and_reject_bad_arguments_before_any_device_work():
    lib = _lib()
    sz = lib.sorsvd_products_workspace_size
    sz.argtypes = [C.c_int64, C.c_int]
    sz.restype = C.c_size_t
    # the operands are the caller's: the workspace holds per-CTA partials and
    # l x l matrices, so it grows with l, not with the rows past one wave
    assert sz(65536, 266) >= sz(64, 266) > 0
    assert sz(4096, 266) > sz(4096, 32) > 0
    assert sz(4096, 266) % 256 == 0
    assert sz(0, 10) == 0 and sz(100, 0) == 0 and sz(1000, 321) == 0
    g = lib.sorsvd_gram
    g.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int64,
                  C.c_void_p, C.c_size_t, C.c_void_p]
    x = 0x1000
    assert g(None, 64, None, 0, 64, 8, x, 8, x, 1 << 20, None) == 1
    assert g(x, 63, None, 0, 64, 8, x, 8, x, 1 << 20, None) == 1      # ldx < rows
    assert g(x, 66, None, 0, 64, 8, x, 8, x, 1 << 20, None) == 1      # ldx not a multiple of 4
    assert g(x + 4, 64, None, 0, 64, 8, x, 8, x, 1 << 20, None) == 1  # X not 16-byte aligned
    assert g(x, 64, x + 8, 64, 64, 8, x, 8, x, 1 << 20, None) == 1    # Y not 16-byte aligned
    assert g(x, 64, None, 0, 64, 8, x, 7, x, 1 << 20, None) == 1      # ldg < l
    assert g(x, 400, None, 0, 400, 321, x, 321, x, 1 << 30, None) == 8  # beyond SORSVD_MAX_L
    assert g(x, 64, None, 0, 64, 8, x, 8, x, 16, None) == 7           # workspace too small
    a = lib.sorsvd_apply
    a.argtypes = [C.c_void_p, C.c_int64, C.c_int, C.c_int64, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p,
                  C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p]
    assert a(x, 64, 8, 64, None, 8, 8, 0, x, 64, x, 1 << 20, None) == 1    # no B
    assert a(x, 64, 8, 64, x, 7, 8, 0, x, 64, x, 1 << 20, None) == 1       # ldb < K
    assert a(x, 64, 8, 64, x, 8, 8, 0, x, 63, x, 1 << 20, None) == 1       # ldy < rows
    assert a(x, 64, 8, 66, x, 8, 8, 0, x, 64, x, 1 << 20, None) == 1       # ldx not a multiple of 4
    assert a(x, 64, 8, 64, x, 8, 321, 0, x, 64, x, 1 << 30, None) == 8     # N beyond SORSVD_MAX_L
    assert a(x, 64, 8, 64, x, 8, 8, 0, x, 64, x + 8, 1 << 20, None) == 7   # workspace misaligned


def test_stage_entry_points_reject_bad_arguments_before_any_device_work():
    lib = _lib()
    x = 0x1000
    gs = lib.sorsvd_gaussian
    gs.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_int, C.c_void_p]
    assert gs(None, 10, 3, 10, 0, 0, 1, None) == 1
    assert gs(x, 10, 3, 9, 0, 0, 1, None) == 1                    # ld < rows
    assert gs(x, -1, 3, 10, 0, 0, 1, None) == 1
    assert gs(x, 10, 3, 10, 0, 0, 9, None) == 2                   # unknown dtype
    ch = lib.sorsvd_chol_inv
    ch.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    assert ch(None, 10, 0.0, 1, x, x, None) == 1
    assert ch(x, 0, 0.0, 1, x, x, None) == 1
    assert ch(x, 10, -1.0, 1, x, x, None) == 1                    # negative shift
    assert ch(x, 10, float("nan"), 1, x, x, None) == 1
    assert ch(x, 225, 0.0, 0, x, x, None) == 8                    # beyond SORSVD_MAX_L_F64
    assert ch(x, 10, 0.0, 9, x, x, None) == 2
    pp = lib.sorsvd_power_pass
    pp.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_int,
                   C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p]
    assert pp(None, 100, 80, 100, 1, x, 80, 10, x, 100, x, 80, x, 1 << 20, None) == 1
    assert pp(x, 100, 80, 99, 1, x, 80, 10, x, 100, x, 80, x, 1 << 20, None) == 1    # lda < m
    assert pp(x, 100, 80, 100, 1, x, 79, 10, x, 100, x, 80, x, 1 << 20, None) == 1   # ldx < n
    assert pp(x, 100, 80, 100, 1, x, 80, 81, x, 100, x, 80, x, 1 << 20, None) == 8   # l > min(m, n)
    assert pp(x, 100, 80, 100, 1, x, 80, 10, x, 100, x, 80, None, 0, None) == 7      # no workspace
    assert pp(x, 100, 80, 100, 9, x, 80, 10, x, 100, x, 80, x, 1 << 20, None) == 2
    co = lib.sorsvd_core
    co.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_uint, C.c_void_p, C.c_int64,
                   C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p]
    assert co(x, 100, 80, 100, 1, 0, None, 100, x, 80, 10, x, 10, x, 1 << 20, None) == 1
    assert co(x, 100, 80, 100, 1, 0, x, 100, x, 80, 10, x, 9, x, 1 << 20, None) == 1    # ldm < l
    assert co(x, 100, 80, 100, 1, 0x40, x, 100, x, 80, 10, x, 10, x, 1 << 20, None) == 1  # flag not of the core
    assert co(x, 100, 80, 100, 1, 0, x, 100, x, 80, 10, x, 10, None, 0, None) == 7      # no workspace
