"""The paper's comparison methods on the library's kernels (Sec. II): the
randomized SVD R-SVD (Algorithm 1, SORSVD_FLAG_RSVD) and the two-sided
randomized SVD TSR-SVD (Algorithm 2, SORSVD_FLAG_TSR), through the C ABI,
against the oracle's rsvd / tsrsvd on the same seeded input and test
matrices (the gates of the SOR-SVD parity tests: |r_gpu - r_oracle| <= tol
and max_j |S_gpu,j - S_oracle,j| / S_oracle,1 <= tol, tol = 1e-10 binary64,
1e-5 fp32, 1e-2 bf16), plus exact recovery of low-rank inputs and the
argument checks of the method flags."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1804_00462_gb300 import inputs  # noqa: E402

TOL = {"f64": 1e-10, "f32": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def nat():
    from paper_1804_00462_gb300 import native
    return native


def cuda_colmajor(store, dtype):
    t = np.ascontiguousarray(store.T)
    if dtype == "bf16":
        x = torch.from_numpy(t.view(np.int16)).cuda().view(torch.bfloat16)
    else:
        x = torch.from_numpy(t).cuda()
    return x.T


def gates(exact, got, ref):
    nA = np.linalg.norm(exact)
    U, S, V = (x.detach().double().cpu().numpy() for x in got)
    Uo, So, Vo = ref
    r_gpu = oracle.recon_error_fro(exact, U, S, V) / nA
    r_orc = oracle.recon_error_fro(exact, Uo, So, Vo) / nA
    ds = float(np.max(np.abs(S - So)) / So[0])
    return r_gpu, r_orc, ds


@pytest.mark.parametrize("dt,m,n,k,p,q", [("f64", 400, 300, 20, 5, 1), ("f64", 260, 500, 12, 8, 0),
                                          ("f32", 2000, 1200, 40, 10, 1), ("f32", 1500, 900, 100, 10, 2),
                                          ("bf16", 2048, 1024, 32, 8, 2)])
def test_rsvd_matches_oracle(nat, dt, m, n, k, p, q):
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 30.0), seed=m + n + q)
    store, exact = inputs.to_storage(A64, dt)
    got = nat.run(cuda_colmajor(store, dt), k, p, q, seed=5, dtype=dt, flags=nat.FLAG_RSVD, check=True)
    torch.cuda.synchronize()
    ref = oracle.rsvd(exact, k, p, q, 5, omega_dtype=dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= TOL[dt] and ds <= TOL[dt], (r_gpu, r_orc, ds)
    ey = oracle.eckart_young(s, k)[1] / np.linalg.norm(exact)
    assert r_gpu >= ey * (1 - 1e-6)


def test_rsvd_equals_sorsvd_on_the_gpu(nat):
    # in exact arithmetic R-SVD's rank-k approximation is SOR-SVD's for the
    # same Omega and q (the rows of B = Q1^T A lie in range(Q2))
    A64 = inputs.spectral(500, 350, inputs.sigma_poly(350, 1.0), seed=3)[0]
    A = cuda_colmajor(np.asfortranarray(A64), "f64")
    U1, S1, V1 = nat.run(A, 15, 5, 1, seed=2, dtype="f64", flags=nat.FLAG_RSVD, check=True)
    U2, S2, V2 = nat.run(A, 15, 5, 1, seed=2, dtype="f64", check=True)
    torch.cuda.synchronize()
    a1 = (U1 * S1[None, :]) @ V1.T
    a2 = (U2 * S2[None, :]) @ V2.T
    assert (torch.linalg.norm(a1 - a2) / torch.linalg.norm(a2)).item() <= 1e-10
    assert torch.allclose(S1, S2, rtol=1e-10, atol=0)


@pytest.mark.parametrize("dt,m,n,k,p", [("f64", 400, 300, 20, 5), ("f64", 200, 450, 10, 6),
                                        ("f32", 1500, 1000, 30, 10), ("bf16", 2048, 1024, 32, 8)])
def test_tsr_matches_oracle(nat, dt, m, n, k, p):
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 10.0), seed=m + 2 * n)
    store, exact = inputs.to_storage(A64, dt)
    got = nat.run(cuda_colmajor(store, dt), k, p, 0, seed=7, dtype=dt, flags=nat.FLAG_TSR, check=True)
    torch.cuda.synchronize()
    ref = oracle.tsrsvd(exact, k, p, 7, omega_dtype=dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    # B_approx multiplies by (Q2^T Psi1)^+: rounding is amplified by its
    # condition number (a Gaussian l x l matrix: a few tens here)
    tol = {"f64": 1e-9, "f32": 1e-4, "bf16": 1e-2}[dt]
    assert abs(r_gpu - r_orc) <= tol and ds <= tol, (r_gpu, r_orc, ds)


@pytest.mark.parametrize("dt", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("method", ["rsvd", "tsr"])
def test_methods_recover_low_rank(nat, dt, method):
    m, n, r, k, p = 700, 500, 12, 12, 6
    A64 = inputs.exact_rank(m, n, r, seed=4)
    store, exact = inputs.to_storage(A64, dt)
    flags = nat.FLAG_RSVD if method == "rsvd" else nat.FLAG_TSR
    U, S, V = nat.run(cuda_colmajor(store, dt), k, p, 0 if method == "tsr" else 1, seed=3, dtype=dt, flags=flags,
                      check=True)
    torch.cuda.synchronize()
    Ah = ((U * S[None, :]) @ V.T).double().cpu().numpy()
    rel = np.linalg.norm(exact - Ah) / np.linalg.norm(exact)
    bound = {"f64": 1e-11, "f32": 1e-5, "bf16": 1e-2}[dt]
    if method == "tsr" and dt == "f32":
        # B_approx = Q1^T Y1 (Q2^T Psi1)^+ amplifies the fp32 rounding of its
        # factors by cond(Q2^T Psi1), that of a Gaussian l x l matrix
        bound = 1e-4
    if method == "tsr" and dt == "bf16":
        # the bf16 copy of a rank-r matrix is rank r plus its rounding (about
        # 2e-3 of |A|), and Algorithm 2 recovers only inputs of rank <= l:
        # (Q2^T Psi1)^+ amplifies that tail (the oracle's own error on the
        # same stored input is near 8e-2), so the GPU result is held to the
        # oracle's error on that input instead of to zero
        Uo, So, Vo = oracle.tsrsvd(exact, k, p, 3, omega_dtype=dt)
        rel_o = np.linalg.norm(exact - (Uo * So[None, :]) @ Vo.T) / np.linalg.norm(exact)
        assert abs(rel - rel_o) <= TOL[dt], (rel, rel_o)
        return
    assert rel <= bound, (method, dt, rel)


def test_method_flag_combinations_are_rejected(nat):
    from paper_1804_00462_gb300.native import _lib
    A = torch.zeros(64, 48, dtype=torch.float64, device="cuda").T.contiguous().T
    U = torch.zeros(48, 64, dtype=torch.float64, device="cuda").T
    V = torch.zeros(8, 48, dtype=torch.float64, device="cuda").T
    S = torch.zeros(8, dtype=torch.float64, device="cuda")
    U = torch.zeros(8, 64, dtype=torch.float64, device="cuda").T
    ws = nat.alloc_workspace(64, 48, 8, 4, "f64", nat.FLAG_TWO_PASS)

    def call(q, flags):
        return _lib.sorsvd_run(A.data_ptr(), 64, 48, 64, 8, 4, q, 1, 0, flags, U.data_ptr(), 64, S.data_ptr(),
                               V.data_ptr(), 48, ws.data_ptr(), ws.numel(), None)
    assert call(1, nat.FLAG_TSR) == 1                          # TSR is one round (q = 0)
    assert call(0, nat.FLAG_RSVD | nat.FLAG_TSR) == 1
    assert call(0, nat.FLAG_RSVD | nat.FLAG_TWO_PASS) == 1
    assert call(1, nat.FLAG_RSVD | nat.FLAG_LITERAL_POWER) == 1
    assert call(0, nat.FLAG_TSR | nat.FLAG_LITERAL_POWER) == 1
    assert call(0, nat.FLAG_TSR) == 0
    assert call(1, nat.FLAG_RSVD) == 0
    torch.cuda.synchronize()
