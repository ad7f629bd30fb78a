"""Parity of the CUDA path (through the C ABI) with the binary64 CPU oracle.

Gates (relative Frobenius reconstruction error r = ||A - U S V^T||_F / ||A||_F
and singular values, on the same seeded input and the same Omega):
  |r_gpu - r_oracle| <= tol  and  max_j |S_gpu_j - S_oracle_j| / S_oracle_1 <= tol
with tol = 1e-10 (F64), 1e-5 (F32 / TF32-free fp32 path), 1e-2 (BF16 / F16
without refinement).  Stage-level checks compare the Gaussian test matrix bit
for bit and the pass / core products element by element.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import philox as oph  # noqa: E402
from paper_1804_00462_gb300 import inputs  # noqa: E402

TOL = {"f64": 1e-10, "f32": 1e-5, "tf32": 1e-2, "bf16": 1e-2, "f16": 1e-2}
TC_ON = os.environ.get("SORSVD_TC", "1") != "0"


def trunc_tf32(x):
    """fp32 value with the low 13 mantissa bits cleared: the operand a TF32
    tensor-core product reads from an fp32 container."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    return (a.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_00462_gb300 import native
    return native


def cuda_colmajor(store: np.ndarray, dtype: str):
    """Fortran-ordered numpy storage -> column-major CUDA tensor (m x n)."""
    t = np.ascontiguousarray(store.T)
    if dtype == "bf16":
        x = torch.from_numpy(t.view(np.int16)).cuda().view(torch.bfloat16)
    else:
        x = torch.from_numpy(t).cuda()
    return x.T


def to_np(x):
    return x.detach().double().cpu().numpy()


def gates(exact, got, ref):
    nA = np.linalg.norm(exact)
    U, S, V = (to_np(t) for t in got)
    Uo, So, Vo = ref
    r_gpu = oracle.recon_error_fro(exact, U, S, V) / nA
    r_orc = oracle.recon_error_fro(exact, Uo, So, Vo) / nA
    ds = float(np.max(np.abs(S - So)) / So[0]) if So[0] > 0 else float(np.max(np.abs(S)))
    return r_gpu, r_orc, ds


def subspace_sin(Y, X, C, j):
    """sin of the largest principal angle between the spans of the first j
    columns of Y and of the orthonormal basis X (C = X^T Y): the spectral
    norm of the residual Y_j - X_j X_j^T Y_j, formed explicitly (the form
    sqrt(1 - sigma_min(C_j)^2) cannot resolve angles below ~1e-8)."""
    R = Y[:, :j] - X[:, :j] @ C[:j, :j]
    return float(np.sqrt(max(0.0, float(np.linalg.eigvalsh(R.T @ R)[-1]))))


def leading_gaps(sigma_core, k, tol):
    """Leading j <= k whose relative gap (sigma_j - sigma_{j+1}) / sigma_1 in
    the oracle's core spectrum exceeds 100 tol: there U_j, V_j are
    determined to about tol / gap."""
    s = np.asarray(sigma_core)
    return [(j, (s[j - 1] - s[j]) / s[0]) for j in range(1, k + 1) if (s[j - 1] - s[j]) / s[0] > 100 * tol]


def check_subspaces(got, ref, info, k, tol, factor=10.0, every=1):
    """Davis-Kahan-Wedin form: sin Theta_j <= factor tol / gap_j for the
    leading j with a gap (every `every`-th of them, and the last); returns
    the largest sin Theta seen."""
    U, S, V = (to_np(t) for t in got)
    Uo, So, Vo = ref
    Cu, Cv = Uo.T @ U, Vo.T @ V
    worst = 0.0
    gaps = leading_gaps(info["sigma_core"], k, tol)
    for j, gap in gaps[::every] + gaps[-1:]:
        su, sv = subspace_sin(U, Uo, Cu, j), subspace_sin(V, Vo, Cv, j)
        assert su <= factor * tol / gap and sv <= factor * tol / gap, (j, gap, su, sv)
        worst = max(worst, su, sv)
    return worst


def run_both(nat, A64, k, p, q, seed, dt, flags=0, mode="stabilised"):
    store, exact = inputs.to_storage(A64, dt)
    A = cuda_colmajor(store, dt)
    got = nat.run(A, k, p, q, seed=seed, dtype=dt, flags=flags, check=True)
    torch.cuda.synchronize()
    ref = oracle.sorsvd(exact, k, p, q, seed, omega_dtype=dt, mode=mode)
    return exact, got, ref


# ---------------------------------------------------------------------------
# stage 1: Omega
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rows,cols", [(1, 1), (7, 3), (333, 27), (1000, 25), (10000, 110)])
@pytest.mark.parametrize("dt", ["f64", "f32", "bf16", "f16"])
def test_gaussian_bit_exact(nat, rows, cols, dt):
    for seed, sid in ((0, 0), (2**64 - 5, 0), (123456789, 3)):
        g = nat.gaussian(rows, cols, seed, sid, dtype=dt)
        ref = oph.gaussian_matrix(rows, cols, seed, sid, dtype=dt)
        assert np.array_equal(to_np(g), ref), (rows, cols, dt, seed)


def test_gaussian_leading_dimension(nat):
    rows, cols, ld = 37, 5, 50
    buf = torch.full((cols, ld), 7.0, dtype=torch.float64, device="cuda")
    r = nat.lib.sorsvd_gaussian(buf.data_ptr(), rows, cols, ld, 99, 0, nat.F64,
                                torch.cuda.current_stream().cuda_stream)
    assert r == 0
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.array_equal(b[:, :rows].T, oph.gaussian_matrix(rows, cols, 99))
    assert np.all(b[:, rows:] == 7.0)


# ---------------------------------------------------------------------------
# stage 2: power pass T1 = A X, T2 = A^T T1
# ---------------------------------------------------------------------------

def elem_tol(dt, K, tc):
    """Componentwise bound |C_gpu - C| <= tol (|A| |X|) of a product over K
    terms, from how each path rounds (u = 2^-24 unit roundoff of fp32):
    CUDA cores (binary64 or fp32 FMA, split-K partials): 2 K u of the type.
    Tensor cores: every MMA (8 TF32 / 16 BF16-FP16 products) adds into the
    fp32 accumulator with at most one truncation, <= 2^-23 of the partial
    (counted twice for the internal adds); partial sums of split tiles
    (<= one per CTA, 152) and drained fills are fp32 round-to-nearest.
    Split TF32 (F32): the operands enter as hi + lo with A's lo truncated
    to TF32 (2^-20), B's lo truncated (2^-21) and lo*lo dropped (2^-21):
    2^-19 per product; the hi*hi fills drain every 16 MMAs."""
    if not tc:
        return 2.0 * K * (2.0 ** -53 if dt == "f64" else 2.0 ** -24)
    parts = 152 * 2.0 ** -24
    if dt == "f32":
        return 2.0 ** -19 + 2 * 16 * 2.0 ** -23 + (-(-K // 128) + 152) * 2.0 ** -24
    per_mma = 8 if dt == "tf32" else 16
    return 2 * (-(-K // per_mma)) * 2.0 ** -23 + parts


def max_elem_ratio(C, Cref, absA, absX):
    """max_ij |C - Cref|_ij / (|A| |X|)_ij."""
    bound = absA @ absX
    return float(np.max(np.abs(C - Cref) / np.maximum(bound, 1e-300)))


@pytest.mark.parametrize("dt", ["f64", "f32", "tf32", "bf16", "f16"])
@pytest.mark.parametrize("m,n,k,p", [(333, 517, 20, 7), (1025, 130, 60, 4), (129, 2049, 9, 1), (4096, 768, 100, 12),
                                     (1000, 360, 27, 5), (2048, 4096, 256, 10), (640, 96, 32, 0),
                                     (1500, 700, 100, 28),
                                     # 16-bit sketches wider than 128 columns run on CTA pairs:
                                     # one N-chunk (l = 160, 200, 256), two (l = 300: the last
                                     # chunk narrower than its box), ragged and tiny M (the
                                     # second CTA's rows out of range), split tiles
                                     (1000, 517, 150, 10), (250, 1030, 190, 10), (3000, 2000, 290, 10),
                                     (70000, 300, 250, 6)])
def test_power_pass_elementwise(nat, dt, m, n, k, p):
    l = k + p
    if dt == "f64" and l > nat.MAX_L_F64:
        pytest.skip("l beyond the binary64 limit of the small factorisations")
    g = np.random.default_rng(m + n)
    A64 = g.standard_normal((m, n))
    store, exact = inputs.to_storage(A64, dt)
    X64 = g.standard_normal((n, l))
    xd = torch.float64 if dt == "f64" else torch.float32
    X = torch.from_numpy(np.ascontiguousarray(X64.T)).to(xd).cuda().T
    T1, T2 = nat.power_pass(cuda_colmajor(store, dt), X, k, p, dtype=dt)
    torch.cuda.synchronize()
    # the operands the pass multiplies: 16-bit roundings for BF16 / F16;
    # for TF32 on tensor cores the TF32 truncations of the fp32 values (the
    # CUDA-core fallback - TMA needs 16-byte aligned strides - is exact
    # fp32); F32 products are fp32-accurate (split TF32).  fp32 products
    # A X read a transposed copy of A (aligned by the library), so only X's
    # leading dimension n decides.
    fp32c = dt == "tf32"
    esz = 4 if dt in ("f32", "tf32") else 2
    nn_tc = TC_ON and dt != "f64" and ((n * 4) % 16 == 0 if dt in ("f32", "tf32") else (m * esz) % 16 == 0)
    tn_tc = TC_ON and dt != "f64" and (m * esz) % 16 == 0
    t_nn = trunc_tf32 if (fp32c and nn_tc) else (lambda x: x)
    t_tn = trunc_tf32 if (fp32c and tn_tc) else (lambda x: x)
    Xr = oph.round_to(to_np(X), dt)
    T1o = t_nn(exact) @ t_nn(Xr)
    T2o = t_tn(exact).T @ t_tn(oph.round_to(T1o, dt))
    T1g, T2g = to_np(T1), to_np(T2)
    e1 = np.linalg.norm(T1g - T1o) / np.linalg.norm(T1o)
    e2 = np.linalg.norm(T2g - T2o) / np.linalg.norm(T2o)
    # norm-wise: the element bounds below over random signs; F32's split
    # products carry ~1e-6 relative error whatever the length of the sum
    # (drained fills, see elem_tol)
    tol1 = {"f64": 1e-14, "f32": 3e-6, "tf32": 1e-4, "bf16": 2e-3, "f16": 1e-3}[dt]
    tol2 = {"f64": 1e-14, "f32": 4e-6, "tf32": 1e-4, "bf16": 2e-3, "f16": 1e-3}[dt]
    assert e1 <= tol1 and e2 <= tol2, (e1, e2)
    # element by element against the componentwise bound of each product
    # (T2 against the product of the kernel's own T1, rounded as the pass
    # rounds it): a misplaced or stale element is off by ~|C_ij| ~ sqrt(K),
    # far above tol (|A| |X|)_ij
    aA = np.abs(t_nn(exact))
    r1 = max_elem_ratio(T1g, T1o, aA, np.abs(t_nn(Xr)))
    T1r = t_tn(oph.round_to(T1g, dt))
    r2 = max_elem_ratio(T2g, t_tn(exact).T @ T1r, np.abs(t_tn(exact)).T, np.abs(T1r))
    assert r1 <= elem_tol(dt, n, nn_tc) and r2 <= elem_tol(dt, m, tn_tc), (r1, r2)


# ---------------------------------------------------------------------------
# stage 4: core M = Q1^T A Q2
# ---------------------------------------------------------------------------

# REFINE (flags 2): Q2 = hi + lo as two 16-bit operands; the rest of Q2 is
# below 2^-(2p+2) relative (p = 7 bf16 / 10 fp16 fraction bits): 4e-6 bf16,
# 6e-8 fp16 per element, plus the fp32 accumulation
@pytest.mark.parametrize("dt,flags,tol", [("f64", 0, 1e-13), ("f32", 0, 3e-6), ("tf32", 0, 2e-6),
                                          ("bf16", 0, 6e-3), ("bf16", 2, 1e-5), ("f16", 0, 1e-3),
                                          ("f16", 2, 2e-6)])
def test_core_elementwise(nat, dt, flags, tol):
    m, n, k, p = 700, 300, 30, 5
    l = k + p
    g = np.random.default_rng(5)
    store, exact = inputs.to_storage(g.standard_normal((m, n)), dt)
    Q1, _ = np.linalg.qr(g.standard_normal((m, l)))
    Q2, _ = np.linalg.qr(g.standard_normal((n, l)))
    qd = torch.float64 if dt == "f64" else torch.float32
    tq1 = torch.from_numpy(np.ascontiguousarray(Q1.T)).to(qd).cuda().T
    tq2 = torch.from_numpy(np.ascontiguousarray(Q2.T)).to(qd).cuda().T
    M = nat.core(cuda_colmajor(store, dt), tq1, tq2, k, p, dtype=dt, flags=flags)
    torch.cuda.synchronize()
    tc = TC_ON and dt != "f64"
    Aop = trunc_tf32(exact) if dt == "tf32" and tc else exact
    Q2op = trunc_tf32(to_np(tq2)) if dt == "tf32" and tc else to_np(tq2)
    Mo = to_np(tq1).T @ (Aop @ Q2op)
    err = np.linalg.norm(to_np(M) - Mo) / np.linalg.norm(Mo)
    assert err <= tol, err
    # element by element: |M - Mo| <= t (|Q1|^T |A| |Q2|) with t the bound of
    # the pass W = A Q2 (K = n), the fp32 Gram Q1^T W (K = m) and the 16-bit
    # rounding of Q2 (REFINE: of what hi + lo leaves, 2^-(2p+2))
    rnd = {"bf16": (2.0 ** -9, 2.0 ** -17), "f16": (2.0 ** -11, 2.0 ** -22)}.get(dt, (0.0, 0.0))[flags == 2]
    t = rnd + (2 if flags == 2 else 1) * elem_tol(dt if dt != "f64" else "f64", n, tc) + \
        (2 * m * 2.0 ** -53 if dt == "f64" else 2 * m * 2.0 ** -24)
    bound = np.abs(to_np(tq1)).T @ (np.abs(Aop) @ np.abs(Q2op))
    assert float(np.max(np.abs(to_np(M) - Mo) / bound)) <= t


# ---------------------------------------------------------------------------
# whole path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("q", [0, 1])
def test_run_cfg1_f64(nat, q):
    A64, s, _, _ = inputs.cfg1(seed=0)
    store, exact = inputs.to_storage(A64, "f64")
    got = nat.run(cuda_colmajor(store, "f64"), 20, 5, q, seed=0, dtype="f64", check=True)
    torch.cuda.synchronize()
    Uo, So, Vo, info = oracle.sorsvd(exact, 20, 5, q, 0, omega_dtype="f64", return_intermediates=True)
    ref = (Uo, So, Vo)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= TOL["f64"] and ds <= TOL["f64"], (r_gpu, r_orc, ds)
    assert r_orc >= oracle.eckart_young(s, 20)[1] / np.linalg.norm(exact) * (1 - 1e-12)
    # the truncation point is well separated (sigma_20 = 1, sigma_21 = 0.79):
    # A_hat = U S V^T is determined, element by element
    U, S, V = (to_np(t) for t in got)
    Ahat, Ahat_o = (U * S) @ V.T, (Uo * So) @ Vo.T
    assert np.max(np.abs(Ahat - Ahat_o)) <= TOL["f64"] * np.max(np.abs(Ahat_o))
    # the leading singular subspaces wherever the core spectrum has a gap
    # (sigma_j = 1 for j <= 20 in A; the sketch's core separates them by
    # 1e-8 .. 0.2): binary64 agreement
    assert len(leading_gaps(info["sigma_core"], 20, TOL["f64"])) >= 1
    assert check_subspaces(got, ref, info, 20, TOL["f64"]) <= 1e-6


def test_run_literal_power_f64(nat):
    A64, s, _, _ = inputs.cfg1(seed=1, n=600)
    exact, got, ref = run_both(nat, A64, 20, 5, 1, 4, "f64", flags=nat.FLAG_LITERAL_POWER, mode="literal")
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= 1e-10 and ds <= 1e-10


@pytest.mark.parametrize("dt", ["f32", "tf32"])
def test_run_noisy_poly_fp32(nat, dt):
    # F32: TF32 sketch passes (they only pick the subspaces) and an fp32
    # core product; TF32: every pass in TF32 (gated like the 16-bit types)
    A64, s, _, _ = inputs.noisy_poly(3000, 1500, 200, 1e-3, seed=2)
    exact, got, ref = run_both(nat, A64, 40, 10, 1, 7, dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= TOL[dt] and ds <= TOL[dt], (r_gpu, r_orc, ds)


@pytest.mark.parametrize("dt", ["bf16", "f16"])
@pytest.mark.parametrize("refine", [False, True])
def test_run_16bit(nat, dt, refine):
    A64, s, _, _ = inputs.spectral(2048, 1024, inputs.sigma_exp(300, 20.0), seed=3)
    flags = nat.FLAG_REFINE if refine else 0
    exact, got, ref = run_both(nat, A64, 32, 8, 2, 1, dt, flags=flags)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= TOL[dt] and ds <= TOL[dt], (r_gpu, r_orc, ds)


@pytest.mark.parametrize("dt,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_run_exact_recovery(nat, dt, tol):
    A64 = inputs.exact_rank(900, 700, 10, seed=8)
    exact, got, ref = run_both(nat, A64, 10, 6, 1, 2, dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert r_gpu <= tol and ds <= tol, (r_gpu, ds)


@pytest.mark.parametrize("m,n,k,p,q", [(300, 200, 1, 0, 0), (150, 150, 100, 50, 1), (200, 900, 17, 3, 2),
                                       (1, 1, 1, 0, 0), (257, 65, 64, 1, 1)])
def test_run_edge_shapes_f64(nat, m, n, k, p, q):
    g = np.random.default_rng(m * n + k)
    A64 = g.standard_normal((m, n)) * np.logspace(0, -4, n)[None, :]
    exact, got, ref = run_both(nat, A64, k, p, q, 5, "f64")
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= 1e-10 and ds <= 1e-10, (r_gpu, r_orc, ds)


def test_run_row_major_input_swaps_factors(nat):
    A64, s, _, _ = inputs.spectral(500, 800, inputs.sigma_poly(500), seed=4)
    At = torch.from_numpy(A64).cuda()                    # row-major m x n
    U, S, V = nat.run(At, 10, 5, 1, seed=3, check=True)
    assert U.shape == (500, 10) and V.shape == (800, 10)
    # the row-major tensor is stored as A^T column-major: the oracle of A^T
    Uo, So, Vo = oracle.sorsvd(A64.T, 10, 5, 1, 3)
    r = oracle.recon_error_fro(A64, to_np(U), to_np(S), to_np(V)) / np.linalg.norm(A64)
    r_o = oracle.recon_error_fro(A64.T, Uo, So, Vo) / np.linalg.norm(A64)
    assert abs(r - r_o) <= 1e-10


def test_device_status_clean_and_sweeps_reported(nat):
    A64, s, _, _ = inputs.cfg1(seed=0, n=400)
    A = cuda_colmajor(np.asfortranarray(A64), "f64")
    ws = nat.alloc_workspace(400, 400, 10, 5, "f64")
    nat.run(A, 10, 5, 1, seed=0, workspace=ws)
    st, info = nat.get_status(ws)
    assert st == 0
    assert 1 <= (info >> 8) & 0xFF < 40


def test_workspace_errors(nat):
    A = torch.zeros(100, 80, dtype=torch.float64, device="cuda").T.contiguous().T
    ws = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(nat.SorsvdError) as e:
        nat.run(A, 5, 5, 0, workspace=ws)
    assert e.value.code == 7


# ---------------------------------------------------------------------------
# full size: the configuration bench.py times (20000 x 10000 fp32, k=100,
# p=10, q=1), whole oracle in binary64 on the host
# ---------------------------------------------------------------------------

def test_run_cfg2_full_size(nat):
    A64, s, _, _ = inputs.cfg2(seed=0)
    store, exact = inputs.to_storage(A64, "f32")
    del A64
    got = nat.run(cuda_colmajor(store, "f32"), 100, 10, 1, seed=0, dtype="f32", check=True)
    torch.cuda.synchronize()
    Uo, So, Vo, info = oracle.sorsvd(exact, 100, 10, 1, 0, omega_dtype="f32", return_intermediates=True)
    ref = (Uo, So, Vo)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    assert abs(r_gpu - r_orc) <= 1e-5 and ds <= 1e-5, (r_gpu, r_orc, ds)
    # the noise bulk (1e-3 N(0,1): singular values ~0.04-0.24) leaves the
    # truncation at k = 100 without a gap, so A_hat is not determined there;
    # the leading singular vectors of the signal (sigma_i = 1/i > 0.24) are
    check_subspaces(got, ref, info, 100, 1e-5)


# ---------------------------------------------------------------------------
# full size: the bf16 65536 x 16384 workload of the bench line (k = 256,
# p = 10, q = 2), plain BF16 and BF16 + REFINE against one binary64 oracle
# solve of the stored matrix
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def cfg3_case():
    A64, s, _, _ = inputs.cfg3(seed=0)
    store, exact = inputs.to_storage(A64, "bf16")
    del A64
    Uo, So, Vo, info = oracle.sorsvd(exact, 256, 10, 2, 0, omega_dtype="bf16", return_intermediates=True)
    return store, exact, (Uo, So, Vo), info


def test_run_cfg3_full_size(nat, cfg3_case):
    store, exact, ref, info = cfg3_case
    A = cuda_colmajor(store, "bf16")
    res = {}
    for refine in (False, True):
        got = nat.run(A, 256, 10, 2, seed=0, dtype="bf16", flags=nat.FLAG_REFINE if refine else 0, check=True)
        torch.cuda.synchronize()
        r_gpu, r_orc, ds = gates(exact, got, ref)
        # the 16-bit class bound on the reconstruction error and the
        # singular values, and on the leading subspaces where they are
        # determined to it
        assert abs(r_gpu - r_orc) <= TOL["bf16"] and ds <= TOL["bf16"], (refine, r_gpu, r_orc, ds)
        check_subspaces(got, ref, info, 256, TOL["bf16"])
        res[refine] = (abs(r_gpu - r_orc), ds)
    del A
    # REFINE (Q2 as a hi + lo bf16 pair in the core, ~16 bits) meets the
    # fp32-class bound 1e-5 on the reconstruction error, and improves on
    # plain BF16 in both the error and the singular values
    assert res[True][0] <= 1e-5, res
    assert res[True][0] < res[False][0] and res[True][1] < res[False][1], res


# ---- CholeskyQR building block ---------------------------------------------
def _rinv_ref(G, shift):
    d = 1.0 / np.sqrt(np.diag(G))
    Gs = G * d[:, None] * d[None, :] + shift * np.eye(G.shape[0])
    L = np.linalg.cholesky(Gs)
    return d[:, None] * np.linalg.inv(L).T


@pytest.mark.parametrize("dt,l", [("f32", 1), ("f32", 7), ("f32", 32), ("f32", 33), ("f32", 64), ("f32", 65),
                                  ("f32", 110), ("f32", 150), ("f32", 200), ("f32", 250), ("f32", 266),
                                  ("f32", 288), ("f32", 300), ("f64", 25), ("f64", 64), ("f64", 150), ("f64", 224)])
def test_chol_inv_matches_numpy(nat, dt, l):
    g = np.random.default_rng(l)
    T = g.standard_normal((2 * l + 3, l)) * np.exp(np.linspace(0, -3, l))[None, :]
    G = T.T @ T
    R, st, info = nat.chol_inv(torch.from_numpy(G).cuda(), 1e-5 if dt == "f32" else 1e-13, dtype=dt)
    torch.cuda.synchronize()
    assert st == 0 and (info & 1) == 0
    Rg = R.double().cpu().numpy()
    Rr = _rinv_ref(G, 1e-5 if dt == "f32" else 1e-13)
    assert np.array_equal(np.tril(Rg, -1), np.zeros_like(Rg))
    tol = 2e-4 if dt == "f32" else 1e-10
    assert np.linalg.norm(Rg - Rr) <= tol * np.linalg.norm(Rr)
    Q = T @ Rg
    assert np.abs(Q.T @ Q - np.eye(l)).max() <= (5e-3 if dt == "f32" else 1e-9)


def test_chol_inv_retry_and_breakdown(nat):
    g = np.random.default_rng(0)
    T = g.standard_normal((50, 20))
    T[:, 5] = T[:, 4]                               # rank deficient: the unshifted factorisation fails
    G = T.T @ T
    R, st, info = nat.chol_inv(torch.from_numpy(G).cuda(), 0.0, dtype="f32")
    torch.cuda.synchronize()
    assert st == 0 and (info & 1) == 1
    assert np.all(np.isfinite(R.cpu().numpy()))
    G[3, 4] = G[4, 3] = np.nan                      # no shift makes this factorisable
    R, st, info = nat.chol_inv(torch.from_numpy(G).cuda(), 0.0, dtype="f32")
    torch.cuda.synchronize()
    assert st == 5                                  # SORSVD_ERR_BREAKDOWN
    assert np.array_equal(R.cpu().numpy(), np.eye(20, dtype=np.float32))


@pytest.mark.parametrize("l", [100, 250])
def test_chol_inv_retry_many_tiles(nat, l):
    # a failed pivot deep in the factorisation restarts it with a larger
    # shift: every tile, including the inverse's tiles formed alongside the
    # factorisation, is rebuilt from the Gram
    g = np.random.default_rng(l)
    T = g.standard_normal((3 * l, l))
    T[:, l - 3] = T[:, l - 40]
    G = T.T @ T
    R, st, info = nat.chol_inv(torch.from_numpy(G).cuda(), 0.0, dtype="f32")
    torch.cuda.synchronize()
    assert st == 0 and (info & 1) == 1
    Rg = R.double().cpu().numpy()
    assert np.all(np.isfinite(Rg)) and np.array_equal(np.tril(Rg, -1), np.zeros_like(Rg))
    # Q = T R: Q^T Q = I - s (G')^{-1} (G' the equilibrated, shifted Gram),
    # so the columns away from the duplicated pair stay orthonormal
    Q = T @ Rg
    keep = [j for j in range(l) if j not in (l - 3, l - 40)]
    E = Q[:, keep].T @ Q[:, keep] - np.eye(l - 2)
    assert np.abs(E).max() <= 0.1


@pytest.mark.parametrize("l,scale", [(1, 0.0), (17, 1e-3), (64, 1e-6), (110, 1e-4), (266, 2e-5), (320, 1e-5)])
def test_polar_inv_near_identity(nat, l, scale):
    # G = D^{1/2} (I + E) D^{1/2}, E symmetric with zero diagonal and
    # ||E||_F <= 0.02: X must equal D^{-1/2} (I + E)^{-1/2}, taken here from
    # an eigendecomposition (independent of the kernel's series), and
    # satisfy X^T G X = I to fp32 level
    g = np.random.default_rng(l)
    E = g.standard_normal((l, l)) * scale
    E = (E + E.T) / 2
    np.fill_diagonal(E, 0.0)
    assert np.linalg.norm(E) <= 0.02
    d = np.exp(g.uniform(-1.0, 1.0, l))
    G = d[:, None] * (np.eye(l) + E) * d[None, :]
    X, ok = nat.polar_inv(torch.from_numpy(G).cuda())
    assert ok == 1
    X = to_np(X)
    w, Qe = np.linalg.eigh(np.eye(l) + E)
    P = (Qe * w ** -0.5) @ Qe.T
    assert np.max(np.abs(X * d[:, None] - P)) <= 1e-6
    assert np.max(np.abs(X.T @ G @ X - np.eye(l))) <= 1e-5


def test_polar_inv_declines_far_from_identity(nat):
    g = np.random.default_rng(3)
    T = g.standard_normal((400, 60))
    T[:, 1] += 0.5 * T[:, 0]                        # columns far from orthonormal
    X, ok = nat.polar_inv(torch.from_numpy(T.T @ T).cuda())
    assert ok == 0


@pytest.mark.parametrize("dt,l", [("f32", 129), ("f32", 200), ("bf16", 266), ("tf32", 288), ("f32", 320)])
def test_run_large_sketch(nat, dt, l):
    """l beyond one SM's shared memory for the Jacobi sweep (cooperative grid
    sweep) and beyond the whole-panel CholeskyQR kernels (tiled Gram and
    product kernels, l > 128); rows 1200 and 700 leave ragged row chunks."""
    k = l - 10
    A64, s, _, _ = inputs.spectral(1200, 700, inputs.sigma_exp(600, 64.0), seed=8)
    exact, got, ref = run_both(nat, A64, k, 10, 1, 2, dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    tol = TOL[dt]
    assert abs(r_gpu - r_orc) <= tol and ds <= tol, (r_gpu, r_orc, ds)
    U, S, V = (to_np(t) for t in got)
    # the sketches are fp32 for every storage type: CholeskyQR3 leaves them
    # orthonormal to fp32 level, and U~, V~ come from the binary64 finish
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-4
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-4


@pytest.mark.parametrize("dt,m,n,k,p,q", [("f32", 4096, 2304, 190, 10, 1), ("bf16", 4096, 2304, 256, 10, 1),
                                          ("tf32", 2048, 4096, 40, 8, 2), ("f16", 3072, 2048, 100, 12, 1),
                                          ("f32", 2560, 2176, 16, 4, 0)])
def test_run_mid_size_wide_sketches(nat, dt, m, n, k, p, q):
    """Sketches of 2048-4096 rows and l up to 266: the split-TF32 passes run
    as column chunks for l > 128, the CholeskyQR factors take their tiled
    form, every pass and product over full tiles and ragged edges."""
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 48.0), seed=m + k)
    exact, got, ref = run_both(nat, A64, k, p, q, 6, dt)
    r_gpu, r_orc, ds = gates(exact, got, ref)
    tol = TOL[dt]
    assert abs(r_gpu - r_orc) <= tol and ds <= tol, (r_gpu, r_orc, ds)
    U, S, V = (to_np(t) for t in got)
    assert np.abs(U.T @ U - np.eye(k)).max() <= 1e-4
    assert np.abs(V.T @ V - np.eye(k)).max() <= 1e-4


@pytest.mark.parametrize("dt,m,n,k,p,q,mode", [("f64", 1000, 600, 20, 5, 0, "stabilised"),
                                               ("f64", 1000, 600, 20, 5, 1, "stabilised"),
                                               ("f64", 700, 500, 15, 5, 1, "literal"),
                                               ("f32", 3000, 1500, 40, 10, 1, "stabilised"),
                                               ("f32", 2560, 2304, 230, 10, 2, "stabilised"),
                                               ("bf16", 2048, 1024, 32, 8, 2, "stabilised"),
                                               ("tf32", 4096, 2048, 100, 12, 1, "stabilised")])
def test_run_two_pass_core(nat, dt, m, n, k, p, q, mode):
    """The two-pass core of Sec. III (M_approx = Q1^T T1 (Q2^T T2_prev)^+, no
    core pass over A) against the oracle's two-pass core on the same loop;
    l = 240 takes the fp32 Cholesky of B B^T (beyond the binary64 limit)."""
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 30.0), seed=m + q)
    flags = nat.FLAG_TWO_PASS | (nat.FLAG_LITERAL_POWER if mode == "literal" else 0)
    store, exact = inputs.to_storage(A64, dt)
    got = nat.run(cuda_colmajor(store, dt), k, p, q, seed=9, dtype=dt, flags=flags, check=True)
    torch.cuda.synchronize()
    ref = oracle.sorsvd(exact, k, p, q, 9, omega_dtype=dt, mode=mode, core="two_pass")
    r_gpu, r_orc, ds = gates(exact, got, ref)
    tol = TOL[dt]
    assert abs(r_gpu - r_orc) <= tol and ds <= tol, (r_gpu, r_orc, ds)
    # the two-pass core approximates the three-pass one: never better than
    # Eckart-Young, and within a few percent of it on this decay
    ey = oracle.eckart_young(s, k)[1] / np.linalg.norm(exact)
    assert ey * (1 - 1e-6) <= r_gpu <= 1.5 * ey
