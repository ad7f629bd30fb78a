"""Python binding of libsorsvd (C ABI in include/sorsvd.h).

Argument marshalling only: every step of SOR-SVD runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (device memory and streams come
from PyTorch).  There is no CPU fallback: if the shared library is missing
the import fails with an explanation.

Matrix layout: the C ABI is column-major.  A torch tensor ``A`` of shape
(m, n) is passed as-is when it is column-major (``A.stride() == (1, lda)``,
e.g. ``At.T`` of a contiguous (n, m) tensor).  A row-major (C-contiguous)
tensor is the column-major storage of A^T; ``run`` then factors A^T and
swaps U and V, which is the same decomposition of A.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

from ._build import LIB

F64, F32, TF32, BF16, F16 = 0, 1, 2, 3, 4
FLAG_LITERAL_POWER = 0x1
FLAG_REFINE = 0x2
FLAG_TWO_PASS = 0x8
FLAG_FIXED_TILES = 0x10
FLAG_RSVD = 0x20
FLAG_TSR = 0x40
MAX_L, MAX_L_F64 = 320, 224

_TORCH_OF = {F64: torch.float64, F32: torch.float32, TF32: torch.float32, BF16: torch.bfloat16,
             F16: torch.float16}
_DT_NAMES = {"f64": F64, "f32": F32, "tf32": TF32, "bf16": BF16, "f16": F16}

if not os.path.exists(LIB):
    raise ImportError(f"libsorsvd.so is not built ({LIB}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
_lib = C.CDLL(LIB)

_i64, _int, _u64, _uint, _vp, _sz = C.c_int64, C.c_int, C.c_uint64, C.c_uint, C.c_void_p, C.c_size_t
_lib.sorsvd_workspace_size.argtypes = [_i64, _i64, _int, _int, _int, _uint]
_lib.sorsvd_workspace_size.restype = _sz
_lib.sorsvd_run.argtypes = [_vp, _i64, _i64, _i64, _int, _int, _int, _u64, _int, _uint,
                            _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]
_lib.sorsvd_run.restype = _int
_lib.sorsvd_run_host.argtypes = [_vp, _i64, _i64, _i64, _int, _int, _int, _u64, _int, _uint,
                                 _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]
_lib.sorsvd_run_host.restype = _int
_lib.sorsvd_streamed_workspace_size.argtypes = [_i64, _i64, _int, _int, _int, _i64]
_lib.sorsvd_streamed_workspace_size.restype = _sz
_lib.sorsvd_run_streamed.argtypes = [_vp, _i64, _i64, _i64, _int, _int, _int, _u64, _int, _i64,
                                     _vp, _i64, _vp, _vp, _i64, _vp, _sz, _vp]
_lib.sorsvd_run_streamed.restype = _int
_lib.sorsvd_get_status.argtypes = [_vp, C.POINTER(_int), C.POINTER(_int), _vp]
_lib.sorsvd_get_status.restype = _int
_lib.sorsvd_set_limits.argtypes = [C.c_longlong, _int]
_lib.sorsvd_set_limits.restype = _int
_lib.sorsvd_status_string.argtypes = [_int]
_lib.sorsvd_status_string.restype = C.c_char_p
_lib.sorsvd_gaussian.argtypes = [_vp, _i64, _i64, _i64, _u64, _u64, _int, _vp]
_lib.sorsvd_gaussian.restype = _int
_lib.sorsvd_power_pass.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _i64, _int, _vp, _i64, _vp, _i64,
                                   _vp, _sz, _vp]
_lib.sorsvd_power_pass.restype = _int
_lib.sorsvd_core.argtypes = [_vp, _i64, _i64, _i64, _int, _uint, _vp, _i64, _vp, _i64, _int, _vp, _i64,
                             _vp, _sz, _vp]
_lib.sorsvd_core.restype = _int

_lib.sorsvd_chol_inv.argtypes = [_vp, _int, C.c_double, _int, _vp, _vp, _vp]
_lib.sorsvd_chol_inv.restype = _int
_lib.sorsvd_polar_inv.argtypes = [_vp, _int, _vp, _vp, _vp, _sz, _vp]
_lib.sorsvd_polar_inv.restype = _int
_lib.sorsvd_products_workspace_size.argtypes = [_i64, _int]
_lib.sorsvd_products_workspace_size.restype = _sz
_lib.sorsvd_gram.argtypes = [_vp, _i64, _vp, _i64, _i64, _int, _vp, _i64, _vp, _sz, _vp]
_lib.sorsvd_gram.restype = _int
_lib.sorsvd_apply.argtypes = [_vp, _i64, _int, _i64, _vp, _i64, _int, _int, _vp, _i64, _vp, _sz, _vp]
_lib.sorsvd_apply.restype = _int

lib = _lib


class SorsvdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (status {code})")


def status_string(code: int) -> str:
    return _lib.sorsvd_status_string(int(code)).decode()


def _check(code: int, where: str):
    if code != 0:
        raise SorsvdError(code, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def dtype_code(dtype) -> int:
    if isinstance(dtype, int):
        return dtype
    if isinstance(dtype, str):
        return _DT_NAMES[dtype]
    for code, td in ((F64, torch.float64), (F32, torch.float32), (BF16, torch.bfloat16), (F16, torch.float16)):
        if dtype == td:
            return code
    raise ValueError(f"unsupported dtype {dtype}")


def out_dtype(code: int):
    return torch.float64 if code == F64 else torch.float32


def workspace_size(m: int, n: int, k: int, p: int, dtype, flags: int = 0) -> int:
    return int(_lib.sorsvd_workspace_size(m, n, k, p, dtype_code(dtype), flags))


def alloc_workspace(m: int, n: int, k: int, p: int, dtype, flags: int = 0, device=None) -> torch.Tensor:
    nb = workspace_size(m, n, k, p, dtype, flags)
    if nb == 0:
        raise SorsvdError(1, "sorsvd_workspace_size")
    return torch.empty(nb, dtype=torch.uint8, device=device or "cuda")


def _colmajor(A: torch.Tensor):
    """(ptr, rows, cols, ld, transposed) of a 2-D CUDA tensor."""
    if A.dim() != 2 or not A.is_cuda:
        raise ValueError("expected a 2-D CUDA tensor")
    r, c = A.shape
    s0, s1 = A.stride()
    if s0 == 1 and (s1 >= max(r, 1) or c == 1):
        return A.data_ptr(), r, c, max(s1, r), False
    if s1 == 1 and (s0 >= max(c, 1) or r == 1):
        return A.data_ptr(), c, r, max(s0, c), True
    raise ValueError("A must be column-major or row-major with unit inner stride")


def colmajor_empty(rows: int, cols: int, dtype, device) -> torch.Tensor:
    return torch.empty(cols, rows, dtype=dtype, device=device).T


def run(A: torch.Tensor, k: int, p: int, q: int, seed: int = 0, dtype=None, flags: int = 0,
        workspace: torch.Tensor | None = None, stream=None, out=None, check: bool = False):
    """Rank-k SOR-SVD of A (Algorithm 3).  Returns (U m x k, S k, V n x k)."""
    ptr, m, n, lda, trans = _colmajor(A)
    code = dtype_code(dtype if dtype is not None else A.dtype)
    if _TORCH_OF[code] != A.dtype:
        raise ValueError(f"dtype code {code} does not match tensor dtype {A.dtype}")
    od = out_dtype(code)
    if out is None:
        U = colmajor_empty(m, k, od, A.device)
        S = torch.empty(k, dtype=od, device=A.device)
        V = colmajor_empty(n, k, od, A.device)
    else:
        U, S, V = out
        if trans:
            U, V = V, U
    if workspace is None:
        workspace = alloc_workspace(m, n, k, p, code, flags, A.device)
    _check(_lib.sorsvd_run(ptr, m, n, lda, k, p, q, seed & 0xFFFFFFFFFFFFFFFF, code, flags,
                           U.data_ptr(), U.stride(1), S.data_ptr(), V.data_ptr(), V.stride(1),
                           workspace.data_ptr(), workspace.numel(), _stream(stream)), "sorsvd_run")
    if check:
        st, info = get_status(workspace, stream)
        _check(st, "sorsvd_run (device)")
    if trans:
        U, V = V, U
    return U, S, V


FLAG_HOST_IO = 0x4


def _colmajor_host(A: torch.Tensor):
    """(ptr, rows, cols, ld, transposed) of a 2-D CPU tensor."""
    if A.dim() != 2 or A.is_cuda:
        raise ValueError("expected a 2-D host (CPU) tensor")
    r, c = A.shape
    s0, s1 = A.stride()
    if s0 == 1 and (s1 >= max(r, 1) or c == 1):
        return A.data_ptr(), r, c, max(s1, r), False
    if s1 == 1 and (s0 >= max(c, 1) or r == 1):
        return A.data_ptr(), c, r, max(s0, c), True
    raise ValueError("A must be column-major or row-major with unit inner stride")


def run_host(A: torch.Tensor, k: int, p: int, q: int, seed: int = 0, dtype=None, flags: int = 0,
             workspace: torch.Tensor | None = None, stream=None, out=None, device=None):
    """sorsvd_run_host: A and the outputs in host memory (pin them with
    ``pin_memory()`` for asynchronous copies).  Returns host (U, S, V); they
    hold the result once the stream has been synchronised."""
    ptr, m, n, lda, trans = _colmajor_host(A)
    code = dtype_code(dtype if dtype is not None else A.dtype)
    if _TORCH_OF[code] != A.dtype:
        raise ValueError(f"dtype code {code} does not match tensor dtype {A.dtype}")
    od = out_dtype(code)
    if out is None:
        pin = A.is_pinned()
        U = torch.empty(k, m, dtype=od, pin_memory=pin).T
        S = torch.empty(k, dtype=od, pin_memory=pin)
        V = torch.empty(k, n, dtype=od, pin_memory=pin).T
    else:
        U, S, V = out
        if trans:
            U, V = V, U
    if workspace is None:
        workspace = alloc_workspace(m, n, k, p, code, flags | FLAG_HOST_IO, device)
    uptr, um, uk, ldu, ut = _colmajor_host(U)
    vptr, vn, vk, ldv, vt = _colmajor_host(V)
    if ut or vt or um != m or vn != n or uk != k or vk != k or S.is_cuda or S.numel() != k:
        raise ValueError("outputs must be column-major host tensors U m x k, S k, V n x k")
    _check(_lib.sorsvd_run_host(ptr, m, n, lda, k, p, q, seed & 0xFFFFFFFFFFFFFFFF, code, flags,
                                uptr, ldu, S.data_ptr(), vptr, ldv,
                                workspace.data_ptr(), workspace.numel(), _stream(stream)), "sorsvd_run_host")
    if trans:
        U, V = V, U
    return U, S, V


def run_streamed(A: torch.Tensor, k: int, p: int, q: int, seed: int = 0, dtype=None, block_rows: int = 65536,
                 workspace: torch.Tensor | None = None, stream=None, device=None):
    """sorsvd_run_streamed: A stays in host memory (pin it with
    ``pin_memory()`` for asynchronous copies) and every pass streams it to
    the device in blocks of ``block_rows`` rows.  Returns device (U, S, V)
    as ``run`` does."""
    ptr, m, n, lda, trans = _colmajor_host(A)
    if trans:
        raise ValueError("A must be column-major (a transposed view of a row-major tensor)")
    code = dtype_code(dtype if dtype is not None else A.dtype)
    if _TORCH_OF[code] != A.dtype:
        raise ValueError(f"dtype code {code} does not match tensor dtype {A.dtype}")
    dev = torch.device(device or "cuda")
    od = out_dtype(code)
    U = colmajor_empty(m, k, od, dev)
    S = torch.empty(k, dtype=od, device=dev)
    V = colmajor_empty(n, k, od, dev)
    if workspace is None:
        nb = int(_lib.sorsvd_streamed_workspace_size(m, n, k, p, code, block_rows))
        if nb == 0:
            raise SorsvdError(1, "sorsvd_streamed_workspace_size")
        workspace = torch.empty(nb, dtype=torch.uint8, device=dev)
    _check(_lib.sorsvd_run_streamed(ptr, m, n, lda, k, p, q, seed & 0xFFFFFFFFFFFFFFFF, code, block_rows,
                                    U.data_ptr(), U.stride(1), S.data_ptr(), V.data_ptr(), V.stride(1),
                                    workspace.data_ptr(), workspace.numel(), _stream(stream)), "sorsvd_run_streamed")
    return U, S, V


def get_status(workspace: torch.Tensor, stream=None):
    st, info = C.c_int(0), C.c_int(0)
    _check(_lib.sorsvd_get_status(workspace.data_ptr(), C.byref(st), C.byref(info), _stream(stream)),
           "sorsvd_get_status")
    return st.value, info.value


def set_limits(wait_cycles: int = 0, max_sweeps: int = 0):
    """Failure-path limits of later calls (0 restores the defaults)."""
    _check(_lib.sorsvd_set_limits(int(wait_cycles), int(max_sweeps)), "sorsvd_set_limits")


def gaussian(rows: int, cols: int, seed: int, stream_id: int = 0, dtype=F64, device="cuda", stream=None):
    code = dtype_code(dtype)
    out = colmajor_empty(rows, cols, _TORCH_OF[code], device)
    _check(_lib.sorsvd_gaussian(out.data_ptr(), rows, cols, max(rows, 1), seed & 0xFFFFFFFFFFFFFFFF,
                                stream_id, code, _stream(stream)), "sorsvd_gaussian")
    return out


def power_pass(A: torch.Tensor, X: torch.Tensor, k: int, p: int, dtype=None,
               workspace: torch.Tensor | None = None, stream=None):
    """T1 = A X, T2 = A^T T1 for column-major A (m x n) and X (n x l)."""
    ptr, m, n, lda, trans = _colmajor(A)
    if trans:
        raise ValueError("power_pass needs a column-major A")
    code = dtype_code(dtype if dtype is not None else A.dtype)
    l = k + p
    xp, xr, xc, ldx, xt = _colmajor(X)
    if xt or xr != n or xc != l:
        raise ValueError("X must be column-major n x l")
    od = out_dtype(code)
    T1 = colmajor_empty(m, l, od, A.device)
    T2 = colmajor_empty(n, l, od, A.device)
    if workspace is None:
        workspace = alloc_workspace(m, n, k, p, code, 0, A.device)
    _check(_lib.sorsvd_power_pass(ptr, m, n, lda, code, xp, ldx, l, T1.data_ptr(), m, T2.data_ptr(), n,
                                  workspace.data_ptr(), workspace.numel(), _stream(stream)),
           "sorsvd_power_pass")
    return T1, T2


def core(A: torch.Tensor, Q1: torch.Tensor, Q2: torch.Tensor, k: int, p: int, dtype=None, flags: int = 0,
         workspace: torch.Tensor | None = None, stream=None):
    """M = Q1^T A Q2 (binary64, l x l) for column-major A, Q1, Q2."""
    ptr, m, n, lda, trans = _colmajor(A)
    if trans:
        raise ValueError("core needs a column-major A")
    code = dtype_code(dtype if dtype is not None else A.dtype)
    l = k + p
    q1, r1, c1, ld1, t1 = _colmajor(Q1)
    q2, r2, c2, ld2, t2 = _colmajor(Q2)
    if t1 or t2 or (r1, c1, r2, c2) != (m, l, n, l):
        raise ValueError("Q1 (m x l) and Q2 (n x l) must be column-major")
    M = colmajor_empty(l, l, torch.float64, A.device)
    if workspace is None:
        workspace = alloc_workspace(m, n, k, p, code, flags, A.device)
    _check(_lib.sorsvd_core(ptr, m, n, lda, code, flags, q1, ld1, q2, ld2, l, M.data_ptr(), l,
                            workspace.data_ptr(), workspace.numel(), _stream(stream)), "sorsvd_core")
    return M


def chol_inv(G: torch.Tensor, shift_rel: float, dtype=F32, stream=None):
    """R^{-1} of a CholeskyQR step for the binary64 Gram G (l x l CUDA
    tensor).  Returns (Rinv, status, info)."""
    if G.dtype != torch.float64 or G.dim() != 2 or G.shape[0] != G.shape[1]:
        raise ValueError("G must be a square binary64 CUDA tensor")
    l = G.shape[0]
    Gc = G.T.contiguous().T if G.stride(0) != 1 else G
    code = dtype_code(dtype)
    R = colmajor_empty(l, l, out_dtype(code), G.device)
    st = torch.zeros(64, dtype=torch.uint8, device=G.device)
    _check(_lib.sorsvd_chol_inv(Gc.data_ptr(), l, shift_rel, code, R.data_ptr(), st.data_ptr(), _stream(stream)),
           "sorsvd_chol_inv")
    s, info = get_status(st, stream)
    return R, s, info


def polar_inv(G: torch.Tensor, stream=None):
    """Polar factor X = D^{-1/2} (I + E)^{-1/2} of a near-identity binary64
    Gram G (l x l CUDA tensor), fp32.  Returns (X, ok)."""
    if G.dtype != torch.float64 or G.dim() != 2 or G.shape[0] != G.shape[1]:
        raise ValueError("G must be a square binary64 CUDA tensor")
    l = G.shape[0]
    Gc = G.T.contiguous().T if G.stride(0) != 1 else G
    X = colmajor_empty(l, l, torch.float32, G.device)
    ok = torch.full((1,), -1, dtype=torch.int32, device=G.device)
    nb = 8 * l * l + 8 * ((l + 31) // 32) * l + 4 * l
    scratch = torch.empty(nb, dtype=torch.uint8, device=G.device)
    _check(_lib.sorsvd_polar_inv(Gc.data_ptr(), l, X.data_ptr(), ok.data_ptr(), scratch.data_ptr(), nb,
                                 _stream(stream)), "sorsvd_polar_inv")
    return X, int(ok.item())


def colmajor_f32(X: torch.Tensor, ld: int = 0) -> torch.Tensor:
    """fp32 column-major copy of a 2-D CUDA tensor whose leading dimension is
    a multiple of 4 (ld, when given, at least the rows), as the tall-skinny
    products require."""
    rows, cols = X.shape
    ld = (max(ld, rows) + 3) // 4 * 4
    buf = torch.zeros(cols, ld, dtype=torch.float32, device=X.device)
    buf[:, :rows] = X.T.to(torch.float32)
    return buf.T[:rows]


def _products_ws(rows: int, l: int, device):
    nb = int(_lib.sorsvd_products_workspace_size(rows, l))
    if nb == 0:
        raise SorsvdError(1, "sorsvd_products_workspace_size")
    return torch.empty(nb, dtype=torch.uint8, device=device), nb


def gram(X: torch.Tensor, Y: torch.Tensor = None, stream=None):
    """G = X^T Y (Y = X when omitted; l x l binary64) of column-major fp32
    CUDA tensors with ld % 4 == 0 (colmajor_f32), through sorsvd_gram.
    Returns (G, status)."""
    ptr, rows, l, ld, tr = _colmajor(X)
    if tr or X.dtype != torch.float32:
        raise ValueError("X must be a column-major fp32 tensor")
    yptr, ldy = None, 0
    if Y is not None:
        yptr, yrows, yl, ldy, ytr = _colmajor(Y)
        if ytr or Y.dtype != torch.float32 or (yrows, yl) != (rows, l):
            raise ValueError("Y must be a column-major fp32 tensor shaped like X")
    ws, nb = _products_ws(rows, l, X.device)
    G = colmajor_empty(l, l, torch.float64, X.device)
    _check(_lib.sorsvd_gram(ptr, ld, yptr, ldy, rows, l, G.data_ptr(), l, ws.data_ptr(), nb, _stream(stream)),
           "sorsvd_gram")
    s, _ = get_status(ws, stream)
    return G, s


def apply(X: torch.Tensor, B: torch.Tensor, upper_tri: bool = False, stream=None):
    """Y = X B (fp32) for a column-major fp32 X (ld % 4 == 0, colmajor_f32)
    and a small fp32 B, through sorsvd_apply.  Returns (Y, status)."""
    ptr, rows, K, ld, tr = _colmajor(X)
    if tr or X.dtype != torch.float32:
        raise ValueError("X must be a column-major fp32 tensor")
    if B.dim() != 2 or B.shape[0] != K:
        raise ValueError("B must be K x N")
    N = B.shape[1]
    Bc = B.to(torch.float32).T.contiguous().T
    ws, nb = _products_ws(rows, max(K, N), X.device)
    Y = colmajor_empty(rows, N, torch.float32, X.device)
    _check(_lib.sorsvd_apply(ptr, rows, K, ld, Bc.data_ptr(), K, N, 1 if upper_tri else 0, Y.data_ptr(), rows,
                             ws.data_ptr(), nb, _stream(stream)), "sorsvd_apply")
    s, _ = get_status(ws, stream)
    return Y, s


class BoundsOut(C.Structure):
    """sorsvd_bounds_out of the C header."""
    _fields_ = [("ey_2", C.c_double), ("ey_fro", C.c_double), ("thm5_upper_2", C.c_double),
                ("thm5_upper_fro", C.c_double), ("thm7_upper_2", C.c_double), ("thm7_upper_fro", C.c_double)]


_lib.sorsvd_bounds.argtypes = [C.POINTER(C.c_double), _int, _i64, _int, _int, _int, C.c_double, C.c_double,
                               C.POINTER(BoundsOut), C.POINTER(C.c_double), C.POINTER(C.c_double)]
_lib.sorsvd_bounds.restype = _int


def bounds(sigma, n: int, k: int, p: int, q: int, omega2_norm: float = -1.0, omega1_pinv_norm: float = -1.0):
    """Theorems 4-7 of Sec. IV for the spectrum ``sigma`` (descending, at
    least k + 1 values) through sorsvd_bounds (host code, no GPU).  Returns a
    dict with ey_2, ey_fro, thm5_upper_2 / _fro, thm7_upper_2 / _fro (floats)
    and thm4_lower, thm6_lower (lists of k floats; Theorems 4 and 5 are NaN
    unless both Omega norms are given)."""
    s = [float(v) for v in sigma]
    arr = (C.c_double * len(s))(*s)
    out = BoundsOut()
    t4 = (C.c_double * k)()
    t6 = (C.c_double * k)()
    _check(_lib.sorsvd_bounds(arr, len(s), n, k, p, q, omega2_norm, omega1_pinv_norm, C.byref(out), t4, t6),
           "sorsvd_bounds")
    d = {f: getattr(out, f) for f, _ in BoundsOut._fields_}
    d["thm4_lower"] = list(t4)
    d["thm6_lower"] = list(t6)
    return d


# ---- batched SOR-SVD ----------------------------------------------------------
class Problem(C.Structure):
    """sorsvd_problem of the C header."""
    _fields_ = [("A", _vp), ("m", _i64), ("n", _i64), ("lda", _i64), ("k", _int), ("p", _int), ("q", _int),
                ("seed", _u64), ("U", _vp), ("ldu", _i64), ("S", _vp), ("V", _vp), ("ldv", _i64)]


_lib.sorsvd_batched_workspace_size.argtypes = [C.POINTER(Problem), _int, _int, _uint]
_lib.sorsvd_batched_workspace_size.restype = _sz
_lib.sorsvd_batched_plan_create.argtypes = [C.POINTER(_vp), C.POINTER(Problem), _int, _int, _uint, _int, _vp, _sz,
                                            _vp]
_lib.sorsvd_batched_plan_create.restype = _int
_lib.sorsvd_batched_plan_launch.argtypes = [_vp, _vp]
_lib.sorsvd_batched_plan_launch.restype = _int
_lib.sorsvd_batched_plan_status.argtypes = [_vp, C.POINTER(_int), _vp]
_lib.sorsvd_batched_plan_status.restype = _int
_lib.sorsvd_batched_plan_launches.argtypes = [_vp]
_lib.sorsvd_batched_plan_launches.restype = _int
_lib.sorsvd_batched_plan_tiles.argtypes = [_vp, C.POINTER(_int), _int]
_lib.sorsvd_batched_plan_tiles.restype = _int
_lib.sorsvd_batched_plan_destroy.argtypes = [_vp]
_lib.sorsvd_batched_plan_destroy.restype = None
_lib.sorsvd_run_batched.argtypes = [C.POINTER(Problem), _int, _int, _uint, _vp, _sz, _vp]
_lib.sorsvd_run_batched.restype = _int


def _per(v, n):
    return list(v) if isinstance(v, (list, tuple)) else [v] * n


class BatchedPlan:
    """A batch of SOR-SVD problems (column-major CUDA matrices ``As`` of one
    dtype, per-problem k, p, q, seed) with its outputs and workspace, planned
    once (optionally captured in a CUDA graph) and run by ``launch``.
    ``U[b]`` (m x k), ``S[b]`` (k), ``V[b]`` (n x k) hold problem b's result."""

    def __init__(self, As, ks, p, q, seeds=0, dtype=None, flags: int = 0, use_graph: bool = True, stream=None):
        nb = len(As)
        ks, ps, qs, seeds = _per(ks, nb), _per(p, nb), _per(q, nb), _per(seeds, nb)
        code = dtype_code(dtype if dtype is not None else As[0].dtype)
        od = out_dtype(code)
        self.As = list(As)
        self.U, self.S, self.V = [], [], []
        arr = (Problem * nb)()
        for b, A in enumerate(self.As):
            ptr, m, n, lda, trans = _colmajor(A)
            if trans or A.dtype != _TORCH_OF[code]:
                raise ValueError("batched problems need column-major matrices of the plan's dtype")
            U = colmajor_empty(m, ks[b], od, A.device)
            S = torch.empty(ks[b], dtype=od, device=A.device)
            V = colmajor_empty(n, ks[b], od, A.device)
            self.U.append(U); self.S.append(S); self.V.append(V)
            arr[b] = Problem(ptr, m, n, lda, ks[b], ps[b], qs[b], int(seeds[b]) & 0xFFFFFFFFFFFFFFFF,
                             U.data_ptr(), U.stride(1), S.data_ptr(), V.data_ptr(), V.stride(1))
        need = int(_lib.sorsvd_batched_workspace_size(arr, nb, code, flags))
        if need == 0:
            raise SorsvdError(1, "sorsvd_batched_workspace_size")
        self.workspace = torch.empty(need, dtype=torch.uint8, device=self.As[0].device)
        self.batch = nb
        self._arr = arr
        h = _vp()
        _check(_lib.sorsvd_batched_plan_create(C.byref(h), arr, nb, code, flags, 1 if use_graph else 0,
                                               self.workspace.data_ptr(), need, _stream(stream)),
               "sorsvd_batched_plan_create")
        self._h = h

    def launch(self, stream=None):
        _check(_lib.sorsvd_batched_plan_launch(self._h, _stream(stream)), "sorsvd_batched_plan_launch")

    def status(self, stream=None):
        codes = (_int * self.batch)()
        _check(_lib.sorsvd_batched_plan_status(self._h, codes, _stream(stream)), "sorsvd_batched_plan_status")
        return list(codes)

    @property
    def launches(self) -> int:
        return int(_lib.sorsvd_batched_plan_launches(self._h))

    @property
    def tiles(self):
        """The tile shape picked for each grouped product stage (0: 128 x 64,
        1: 64 x 64, 2: 64 x 32)."""
        n = int(_lib.sorsvd_batched_plan_tiles(self._h, None, 0))
        out = (_int * max(n, 1))()
        _lib.sorsvd_batched_plan_tiles(self._h, out, n)
        return list(out)[:n]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.sorsvd_batched_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batched(As, ks, p, q, seeds=0, dtype=None, flags: int = 0, stream=None):
    """One-shot batched SOR-SVD (no graph); returns [(U, S, V) per problem]."""
    plan = BatchedPlan(As, ks, p, q, seeds, dtype, flags, use_graph=False, stream=stream)
    plan.launch(stream)
    out = list(zip(plan.U, plan.S, plan.V))
    plan.close()
    return out


def batched_workspace_size(problems, dtype, flags: int = 0) -> int:
    """Workspace bytes for a list of (m, n, k, p, q) (no device memory touched)."""
    nb = len(problems)
    arr = (Problem * nb)()
    for b, (m, n, k, p, q) in enumerate(problems):
        arr[b] = Problem(1, m, n, m, k, p, q, 0, 1, m, 1, 1, n)
    return int(_lib.sorsvd_batched_workspace_size(arr, nb, dtype_code(dtype), flags))


# ---- robust PCA ---------------------------------------------------------------
class RpcaProblem(C.Structure):
    """sorsvd_rpca_problem of the C header."""
    _fields_ = [("X", _vp), ("m", _i64), ("n", _i64), ("ldx", _i64),
                ("L", _vp), ("ldl", _i64), ("S", _vp), ("lds", _i64),
                ("norm2", C.c_double), ("seed", _u64)]


RPCA_FINISH_F64 = 0x100
_lib.sorsvd_rpca_workspace_size.argtypes = [C.POINTER(RpcaProblem), _int, _int, _int, _int, _uint]
_lib.sorsvd_rpca_workspace_size.restype = _sz
_lib.sorsvd_rpca.argtypes = [C.POINTER(RpcaProblem), _int, _int, _int, _int, _int, _uint, C.c_double, _int,
                             C.c_double, C.POINTER(_int), C.POINTER(C.c_double), C.POINTER(C.c_double),
                             _vp, _sz, _vp]
_lib.sorsvd_rpca.restype = _int


def _rpca_problems(Xs, Ls, Ss, seeds, norm2s):
    arr = (RpcaProblem * len(Xs))()
    for b, X in enumerate(Xs):
        ptr, m, n, ldx, trans = _colmajor(X)
        if trans or X.dtype != torch.float32:
            raise ValueError("rpca needs column-major fp32 matrices")
        arr[b] = RpcaProblem(ptr, m, n, ldx, Ls[b].data_ptr(), Ls[b].stride(1), Ss[b].data_ptr(),
                             Ss[b].stride(1), float(norm2s[b]), int(seeds[b]) & 0xFFFFFFFFFFFFFFFF)
    return arr


def rpca(Xs, k: int, p: int, q: int, seeds=0, norm2=None, dtype=F32, finish_f64: bool = True,
         tol: float = 1e-7, max_iter: int = 50, rho: float = 1.5, workspace: torch.Tensor | None = None,
         stream=None):
    """Robust PCA (inexact ALM with SOR-SVD, Table 3) of each column-major
    fp32 matrix in ``Xs`` (a tensor or a list).  ``seeds`` / ``norm2``: one
    value or one per problem (norm2 <= 0 or None: estimated on the device).
    ``dtype``: inner SOR-SVD type; ``finish_f64``: switch it to binary64
    near convergence (SORSVD_RPCA_FINISH_F64).
    Returns (Ls, Ss, iters, xi, xi_history) with xi_history a (batch,
    max_iter) CPU tensor (entries past iters[b] are zero)."""
    single = isinstance(Xs, torch.Tensor)
    Xs = [Xs] if single else list(Xs)
    nb = len(Xs)
    seeds = [seeds] * nb if isinstance(seeds, int) else list(seeds)
    norm2s = [0.0 if norm2 is None else norm2] * nb if not isinstance(norm2, (list, tuple)) else list(norm2)
    Ls = [colmajor_empty(X.shape[0], X.shape[1], torch.float32, X.device) for X in Xs]
    Ss = [colmajor_empty(X.shape[0], X.shape[1], torch.float32, X.device) for X in Xs]
    arr = _rpca_problems(Xs, Ls, Ss, seeds, norm2s)
    code = dtype_code(dtype)
    flags = RPCA_FINISH_F64 if finish_f64 else 0
    need = int(_lib.sorsvd_rpca_workspace_size(arr, nb, k, p, code, flags))
    if need == 0:
        raise SorsvdError(1, "sorsvd_rpca_workspace_size")
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=Xs[0].device)
    iters = (_int * nb)()
    xi = (C.c_double * nb)()
    hist = (C.c_double * (nb * max_iter))()
    _check(_lib.sorsvd_rpca(arr, nb, k, p, q, code, flags, tol, max_iter, rho, iters, xi, hist,
                            workspace.data_ptr(), workspace.numel(), _stream(stream)), "sorsvd_rpca")
    xh = torch.tensor(list(hist), dtype=torch.float64).reshape(nb, max_iter)
    if single:
        return Ls[0], Ss[0], iters[0], xi[0], xh[0]
    return Ls, Ss, list(iters), list(xi), xh


def rpca_workspace_size(Xs, k: int, p: int, dtype=F32, norm2=None, finish_f64: bool = True) -> int:
    Xs = [Xs] if isinstance(Xs, torch.Tensor) else list(Xs)
    nb = len(Xs)
    norm2s = [0.0 if norm2 is None else norm2] * nb if not isinstance(norm2, (list, tuple)) else list(norm2)
    arr = _rpca_problems(Xs, Xs, Xs, [0] * nb, norm2s)
    return int(_lib.sorsvd_rpca_workspace_size(arr, nb, k, p, dtype_code(dtype),
                                               RPCA_FINISH_F64 if finish_f64 else 0))


# ---- launch accounting ------------------------------------------------------
NUM_KCLASS = 10
KCLASS_NAMES = ("gaussian", "pass", "core_pass", "small_gemm", "reduce", "chol", "jacobi", "misc", "pass_split",
                "rpca")
_lib.sorsvd_launch_count.argtypes = []
_lib.sorsvd_launch_count.restype = C.c_uint64
_lib.sorsvd_profile_begin.argtypes = [_uint]
_lib.sorsvd_profile_begin.restype = _int
_lib.sorsvd_profile_end.argtypes = [C.POINTER(C.c_double), C.POINTER(_int), _int]
_lib.sorsvd_profile_end.restype = _int


def launch_count() -> int:
    return int(_lib.sorsvd_launch_count())


def profile_begin(classes=KCLASS_NAMES):
    mask = 0
    for c in classes:
        mask |= 1 << KCLASS_NAMES.index(c)
    _check(_lib.sorsvd_profile_begin(mask), "sorsvd_profile_begin")


def profile_end():
    """{class name: (total ms, launches)} of the launches since profile_begin."""
    ms = (C.c_double * NUM_KCLASS)()
    ln = (_int * NUM_KCLASS)()
    _check(_lib.sorsvd_profile_end(ms, ln, NUM_KCLASS), "sorsvd_profile_end")
    return {KCLASS_NAMES[i]: (ms[i], ln[i]) for i in range(NUM_KCLASS)}
