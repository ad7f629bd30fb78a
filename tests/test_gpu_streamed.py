"""Out-of-core SOR-SVD (sorsvd_run_streamed: A in host memory, streamed to
the device in blocks of rows for every pass) through the C ABI: against the
binary64 oracle with the parity gates of the in-core path (|r_gpu - r_oracle|
<= tol and max_j |S_gpu,j - S_oracle,j| / S_oracle,1 <= tol; tol 1e-10
binary64, 1e-5 fp32, 1e-2 bf16), against sorsvd_run on the same input
(A_hat within the dtype's tolerance: only the summation order of
T2 = A^T Q1 differs), for block sizes that divide m, that do not, that hold
all of A, and single rows; pinned and pageable host memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1804_00462_gb300 import inputs  # noqa: E402

TOL = {"f64": 1e-10, "f32": 1e-5, "tf32": 1e-2, "bf16": 1e-2}


@pytest.fixture(scope="module")
def nat():
    from paper_1804_00462_gb300 import native
    return native


def host_colmajor(store, dtype, pin=True):
    t = torch.from_numpy(np.ascontiguousarray(store.T).view(np.int16) if dtype == "bf16" else
                         np.ascontiguousarray(store.T))
    if dtype == "bf16":
        t = t.view(torch.bfloat16)
    if pin:
        t = t.pin_memory()
    return t.T


def ahat(U, S, V):
    return ((U * S[None, :]) @ V.T).double().cpu().numpy()


@pytest.mark.parametrize("dt,m,n,k,p,q,block", [("f64", 600, 400, 20, 5, 1, 256), ("f32", 3000, 1500, 40, 10, 1, 1024),
                                                ("f32", 2500, 1800, 60, 10, 2, 700), ("bf16", 4096, 2048, 32, 8, 2, 1536),
                                                ("tf32", 2000, 1000, 30, 6, 1, 2000)])
def test_streamed_matches_oracle_and_in_core(nat, dt, m, n, k, p, q, block):
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 30.0), seed=m + n)
    store, exact = inputs.to_storage(A64, dt)
    Ah = host_colmajor(store, dt)
    got = nat.run_streamed(Ah, k, p, q, seed=4, dtype=dt, block_rows=block)
    ind = nat.run(Ah.cuda(), k, p, q, seed=4, dtype=dt, check=True)
    torch.cuda.synchronize()
    U, S, V = (x.double().cpu().numpy() for x in got)
    Uo, So, Vo = oracle.sorsvd(exact, k, p, q, 4, omega_dtype=dt)
    nA = np.linalg.norm(exact)
    r_gpu = oracle.recon_error_fro(exact, U, S, V) / nA
    r_orc = oracle.recon_error_fro(exact, Uo, So, Vo) / nA
    ds = float(np.max(np.abs(S - So)) / So[0])
    tol = TOL[dt]
    assert abs(r_gpu - r_orc) <= tol and ds <= tol, (r_gpu, r_orc, ds)
    diff = np.linalg.norm(ahat(*got) - ahat(*ind)) / nA
    assert diff <= tol, diff


@pytest.mark.parametrize("block", [1000, 5000, 1])
def test_block_sizes_and_pageable_memory(nat, block):
    m, n, k, p, q = 1000, 300, 10, 5, 1
    A64 = inputs.exact_rank(m, n, 10, seed=2)
    Ah = host_colmajor(np.asfortranarray(A64), "f64", pin=block != 1)
    U, S, V = nat.run_streamed(Ah, k, p, q, seed=1, dtype="f64", block_rows=block)
    torch.cuda.synchronize()
    rel = np.linalg.norm(A64 - ahat(U, S, V)) / np.linalg.norm(A64)
    assert rel <= 1e-12, rel


def test_streamed_arguments(nat):
    from paper_1804_00462_gb300.native import _lib
    assert int(_lib.sorsvd_streamed_workspace_size(100, 80, 5, 3, 1, 0)) == 0       # block_rows < 1
    assert int(_lib.sorsvd_streamed_workspace_size(100, 80, 5, 3, 1, 32)) > 0
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    A = torch.zeros(80, 100, dtype=torch.float32).T
    U = torch.zeros(5, 100, device="cuda").T
    V = torch.zeros(5, 80, device="cuda").T
    S = torch.zeros(5, device="cuda")
    # workspace too small
    assert _lib.sorsvd_run_streamed(A.data_ptr(), 100, 80, 100, 5, 3, 1, 0, 1, 32, U.data_ptr(), 100, S.data_ptr(),
                                    V.data_ptr(), 80, ws.data_ptr(), ws.numel(), None) == 7
