"""sorsvd_run_noalloc: the entry point for callers that cannot allocate
device memory when they call (it takes its scratch from a library-owned
device array).  Checked through the C ABI against sorsvd_run with a caller
workspace, on two calls in a row (the shared scratch keeps the first call's
contents when the second starts), with the device status word of each call
read back through sorsvd_noalloc_get_status."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1804_00462_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_00462_gb300 import native
    f = native.lib.sorsvd_run_noalloc
    f.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int,
                  C.c_uint, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    f.restype = C.c_int
    g = native.lib.sorsvd_noalloc_get_status
    g.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p]
    g.restype = C.c_int
    return native


def _noalloc_status(nat):
    st, info = C.c_int(-1), C.c_int(-1)
    rc = nat.lib.sorsvd_noalloc_get_status(C.byref(st), C.byref(info), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, nat.status_string(rc)
    return st.value, info.value


def _noalloc(nat, A, k, p, q, seed, code):
    m, n = A.shape
    od = nat.out_dtype(code)
    U = nat.colmajor_empty(m, k, od, "cuda")
    S = torch.empty(k, dtype=od, device="cuda")
    V = nat.colmajor_empty(n, k, od, "cuda")
    rc = nat.lib.sorsvd_run_noalloc(A.data_ptr(), m, n, A.stride(1), k, p, q, seed, code, 0, U.data_ptr(),
                                    U.stride(1), S.data_ptr(), V.data_ptr(), V.stride(1),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == 0, nat.status_string(rc)
    torch.cuda.synchronize()
    return U, S, V


def _rel(A64, U, S, V):
    to = lambda t: t.double().cpu().numpy()
    return oracle.recon_error_fro(A64, to(U), to(S), to(V)) / np.linalg.norm(A64)


def test_noalloc_matches_workspace_entry_point_twice(nat):
    cases = [
        ("f64", *inputs.cfg1(seed=2, n=500)[:1], 20, 5, 1, 7),
        ("f32", *inputs.noisy_poly(1200, 800, 100, 1e-3, seed=3)[:1], 30, 8, 1, 9),
    ]
    for dt, A64, k, p, q, seed in cases:
        code = nat.dtype_code(dt)
        store, exact = inputs.to_storage(A64, dt)
        A = torch.from_numpy(np.ascontiguousarray(store.T)).cuda().T
        Ur, Sr, Vr = nat.run(A, k, p, q, seed=seed, dtype=dt, check=True)
        Un, Sn, Vn = _noalloc(nat, A, k, p, q, seed, code)
        # the device status word of the call (kept in the library's array)
        st, info = _noalloc_status(nat)
        assert st == 0, nat.status_string(st)
        assert (info >> 8) & 0xFF > 0                # Jacobi sweeps of the call
        tol = 1e-10 if dt == "f64" else 1e-5
        assert abs(_rel(exact, Un, Sn, Vn) - _rel(exact, Ur, Sr, Vr)) <= tol
        assert float((Sn.double() - Sr.double()).abs().max() / Sr.double()[0]) <= tol
        # same kernels, same Omega: the two entry points agree bit for bit
        assert torch.equal(Sn, Sr) and torch.equal(Un, Ur) and torch.equal(Vn, Vr)


def test_noalloc_rejects_problems_beyond_its_scratch(nat):
    m, n, k, p = 20000, 10000, 100, 10
    assert nat.workspace_size(m, n, k, p, "f32") > 33554432
    A = torch.empty(n, m, device="cuda").T
    U = nat.colmajor_empty(m, k, torch.float32, "cuda")
    S = torch.empty(k, device="cuda")
    V = nat.colmajor_empty(n, k, torch.float32, "cuda")
    rc = nat.lib.sorsvd_run_noalloc(A.data_ptr(), m, n, m, k, p, 1, 0, nat.F32, 0, U.data_ptr(), m, S.data_ptr(),
                                    V.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    assert rc == 8                                   # SORSVD_ERR_UNSUPPORTED
    rc = nat.lib.sorsvd_run_noalloc(A.data_ptr(), m, n, m - 1, k, p, 1, 0, nat.F32, 0, U.data_ptr(), m,
                                    S.data_ptr(), V.data_ptr(), n, torch.cuda.current_stream().cuda_stream)
    assert rc == 1                                   # SORSVD_ERR_ARG (lda < m)
