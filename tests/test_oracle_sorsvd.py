"""Pins of the oracle's SOR-SVD (Algorithm 3) against what the paper and the
mathematics fix: exact recovery of low-rank inputs, Eckart-Young optimality
(Theorem 1), Thompson interlacing, the Pythagorean split and restricted
optimality of Theorem 2, Gu's projector invariance (Lemma 1: stabilised and
literal power loops agree), the deterministic bounds of Theorems 4-5, the
average bounds of Theorems 6-7, and the values printed in Fig. 4."""
import numpy as np
import pytest

from conftest import golden_rows
from oracle import bounds
from oracle import sor_svd as orc
from oracle.linalg import householder_qr
from paper_1804_00462_gb300 import inputs


def _rel(A, U, S, V):
    return orc.recon_error_fro(A, U, S, V) / np.linalg.norm(A)


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("mode", ["stabilised", "literal"])
def test_exact_recovery_of_rank_r(q, mode):
    A = inputs.exact_rank(300, 200, 12, seed=q)
    U, S, V = orc.sorsvd(A, 12, 4, q, seed=1, mode=mode)
    assert _rel(A, U, S, V) < 1e-12
    assert np.linalg.norm(U.T @ U - np.eye(12)) < 1e-12
    assert np.linalg.norm(V.T @ V - np.eye(12)) < 1e-12


def test_exact_recovery_rank_below_l_and_wide_matrix():
    A = inputs.exact_rank(90, 240, 5, seed=4)          # m < n, rank 5 < k = 8
    U, S, V = orc.sorsvd(A, 8, 4, 1, seed=2)
    assert _rel(A, U, S, V) < 1e-12
    assert np.all(S[5:] < 1e-12 * S[0])


@pytest.mark.parametrize("seed", range(4))
def test_optimality_and_interlacing_tiny(seed):
    g = np.random.default_rng(seed)
    A = g.standard_normal((40, 30)) * np.logspace(0, -3, 30)[None, :]
    s_true = np.linalg.svd(A, compute_uv=False)        # brute force
    k, p = 5, 3
    for q in (0, 1):
        U, S, V = orc.sorsvd(A, k, p, q, seed)
        err = orc.recon_error_fro(A, U, S, V)
        assert err >= orc.eckart_young(s_true, k)[1] * (1 - 1e-12)      # Theorem 1
        assert np.all(S <= s_true[:k] * (1 + 1e-12))                    # Thompson
        s_hat = np.linalg.svd((U * S) @ V.T, compute_uv=False)[:k]
        assert np.allclose(s_hat, S, rtol=1e-12)


def test_theorem2_pythagorean_split_and_restricted_optimality():
    g = np.random.default_rng(8)
    A = g.standard_normal((60, 45))
    k, l = 4, 9
    _, _, _, info = orc.sorsvd(A, k, l - k, 0, seed=3, return_intermediates=True)
    Q1, Q2, M = info["Q1"], info["Q2"], info["M"]
    P = Q1 @ Q1.T @ A @ Q2 @ Q2.T
    Uk, sk, Vkt = np.linalg.svd(M)
    Mk = (Uk[:, :k] * sk[:k]) @ Vkt[:k]
    best = np.linalg.norm(A - Q1 @ Mk @ Q2.T)
    for trial in range(20):
        X = g.standard_normal((l, k)) @ g.standard_normal((k, l))
        lhs = np.linalg.norm(A - Q1 @ X @ Q2.T) ** 2
        rhs = np.linalg.norm(A - P) ** 2 + np.linalg.norm(M - X) ** 2
        assert abs(lhs - rhs) <= 1e-12 * lhs
        assert np.linalg.norm(A - Q1 @ X @ Q2.T) >= best
    U, S, V = orc.sorsvd(A, k, l - k, 0, seed=3)
    assert abs(orc.recon_error_fro(A, U, S, V) - best) <= 1e-12 * best


def test_lemma1_stabilised_equals_literal_cfg1_shape():
    A, s, _, _ = inputs.cfg1(seed=0)
    Ua, Sa, Va = orc.sorsvd(A, 20, 5, 1, seed=0, mode="stabilised")
    Ub, Sb, Vb = orc.sorsvd(A, 20, 5, 1, seed=0, mode="literal")
    Ah_a, Ah_b = (Ua * Sa) @ Va.T, (Ub * Sb) @ Vb.T
    assert np.linalg.norm(Ah_a - Ah_b) <= 1e-10 * np.linalg.norm(A)


def test_fig4_eckart_young_value_is_reproduced():
    rows = golden_rows("fig4_poly_decay.txt")
    s = inputs.sigma_poly(1000)
    ey = orc.eckart_young(s, 10)[1]
    for r in rows:
        assert abs(ey - float(r[1])) <= 1e-15


def test_fig4_sorsvd_errors_in_paper_range():
    rows = {int(r[0]): (float(r[1]), float(r[2]), float(r[3])) for r in golden_rows("fig4_poly_decay.txt")}
    A, s, _, _ = inputs.spectral(1000, 1000, inputs.sigma_poly(1000), seed=0)
    ey = rows[40][0]
    # q = 2, l = 40: paper 0.306866173529286 (excess 6.9e-8 over the SVD line)
    excess = []
    for seed in range(4):
        U, S, V = orc.sorsvd(A, 10, 30, 2, seed)
        excess.append(orc.recon_error_fro(A, U, S, V) / ey - 1)
    assert min(excess) >= -1e-12
    assert np.mean(excess) <= 1e-6
    # q = 0: single draws scatter; compare the seed-mean with the paper's draw
    for l, tol in ((40, 0.05), (30, 0.06), (12, 0.25)):
        errs = []
        for seed in range(4):
            U, S, V = orc.sorsvd(A, 10, l - 10, 0, seed)
            errs.append(orc.recon_error_fro(A, U, S, V))
        assert min(errs) >= ey
        assert abs(np.mean(errs) / rows[l][1] - 1) <= tol


@pytest.mark.parametrize("q", [0, 1, 2])
def test_theorems_4_and_5_hold_per_draw(q):
    # noisy low-rank matrix of Sec. V-A-1 (k = 20) at a smaller order
    n, k = 300, 20
    sig = np.concatenate([np.logspace(0, -2, k), 1e-3 * np.ones(n - k)])
    A, s, U0, V0 = inputs.spectral(n, n, sig, seed=5)
    for l in (22, 30, 40):
        for seed in range(3):
            U, S, V, info = orc.sorsvd(A, k, l - k, q, seed, return_intermediates=True)
            om = info["omega"]
            # Theorem 4 as its proof establishes it: for sigma_j(A Q2 Q2^T)
            lower = bounds.thm4_lower(s, V0, om, k, q)
            Q2 = info["Q2"]
            s_right = np.linalg.svd(A @ Q2 @ Q2.T, compute_uv=False)[:k]
            assert np.all(s_right >= lower * (1 - 1e-12))
            assert np.all(S <= s[:k] * (1 + 1e-12))
            D = A - (U * S) @ V.T
            assert np.linalg.norm(D) <= bounds.thm5_upper(s, V0, om, k, q, "fro") * (1 + 1e-10)
            assert np.linalg.norm(D, 2) <= bounds.thm5_upper(s, V0, om, k, q, "2") * (1 + 1e-10)


@pytest.mark.parametrize("q", [0, 1])
def test_theorems_6_and_7_hold_on_average(q):
    n, k, p = 200, 10, 4
    A, s, _, _ = inputs.spectral(n, n, inputs.sigma_poly(n), seed=2)
    errs_f, errs_2, svs = [], [], []
    for seed in range(20):
        U, S, V = orc.sorsvd(A, k, p, q, seed)
        D = A - (U * S) @ V.T
        errs_f.append(np.linalg.norm(D))
        errs_2.append(np.linalg.norm(D, 2))
        svs.append(S)
    assert np.mean(errs_f) <= bounds.thm7_expected_upper(s, n, k, p, q, "fro")
    assert np.mean(errs_2) <= bounds.thm7_expected_upper(s, n, k, p, q, "2")
    assert np.all(np.mean(svs, axis=0) >= bounds.thm6_expected_lower(s, n, k, p, q))


def test_two_pass_core_recovers_low_rank_and_tracks_three_pass():
    A = inputs.exact_rank(200, 150, 6, seed=3)
    for q in (0, 1):
        U, S, V = orc.sorsvd(A, 6, 4, q, seed=0, core="two_pass")
        assert _rel(A, U, S, V) < 1e-10
    B, s, _, _ = inputs.spectral(300, 300, inputs.sigma_poly(300, 2.0), seed=1)
    e3 = orc.recon_error_fro(B, *orc.sorsvd(B, 10, 10, 1, 0))
    e2 = orc.recon_error_fro(B, *orc.sorsvd(B, 10, 10, 1, 0, core="two_pass"))
    ey = orc.eckart_young(s, 10)[1]
    assert ey <= e3 <= e2 * (1 + 1e-9) and e2 <= 1.5 * ey


def test_flop_count_matches_paper_example_terms():
    # eq. C_SOR-SVD+PM with C_mult = 2mn: at q = 0 the count is 3 passes of
    # 2mnl plus the QR/assembly terms; doubling m and n quadruples the pass term.
    f = orc.flop_count(1000, 1000, 20, 5, 0)
    assert f == 3 * 25 * 2 * 1000 * 1000 + 2 * 25 * 2000 * 45 + 2 * 625 * 1025
    assert orc.flop_count(1000, 1000, 20, 5, 1) - f == 2 * 25 * 2 * 1000 * 1000


class _Counting(np.ndarray):
    """ndarray view that adds 2 r c k to a counter for every r x k by k x c
    matrix product it takes part in (the usual multiply-add count)."""
    flops = [0]

    def __array_ufunc__(self, ufunc, method, *args, **kw):
        plain = [np.asarray(a) if isinstance(a, _Counting) else a for a in args]
        if ufunc is np.matmul and method == "__call__":
            a, b = plain
            _Counting.flops[0] += 2 * a.shape[0] * a.shape[1] * (b.shape[1] if b.ndim == 2 else 1)
        out = getattr(ufunc, method)(*plain, **kw)
        return out.view(_Counting) if isinstance(out, np.ndarray) else out


@pytest.mark.parametrize("m,n,k,p,q", [(60, 40, 3, 2, 0), (50, 70, 4, 3, 1), (80, 30, 5, 5, 2)])
def test_flop_count_equals_the_operations_the_oracle_performs(monkeypatch, m, n, k, p, q):
    # Sec. IV-C prices a QR factorisation or an SVD of an r x c matrix at
    # 2 r c^2 flops and a product with A at C_mult = 2mn per vector.  Run the
    # printed algorithm (literal power loop) with every matrix product, QR
    # and SVD counted at those prices: the total must be eq.
    # (C_SOR-SVD+PM) exactly, so a dropped pass, QR, core or assembly term
    # in flop_count fails here.
    real_qr, real_svd = orc.householder_qr, orc.jacobi_svd

    def qr(T):
        r, c = T.shape
        _Counting.flops[0] += 2 * r * c * c
        Q, R = real_qr(np.asarray(T))
        return Q.view(_Counting), R

    def svd(M):
        r, c = M.shape
        _Counting.flops[0] += 2 * r * c * c
        return real_svd(np.asarray(M))
    monkeypatch.setattr(orc, "householder_qr", qr)
    monkeypatch.setattr(orc, "jacobi_svd", svd)
    A = np.random.default_rng(m).standard_normal((m, n)).view(_Counting)
    _Counting.flops[0] = 0
    orc.sorsvd(A, k, p, q, seed=1, mode="literal")
    assert _Counting.flops[0] == orc.flop_count(m, n, k, p, q)


def test_bounds_at_hand_computed_values():
    # A = diag(2, 1, 1/2, 1/4) (V = I), k = 1, p = 2, l = 3 and
    # Omega = [[2,0,0],[0,1,0],[0,0,1],[0,0,0]]: Omega1 = V1^T Omega = (2 0 0)
    # has sigma_min 2 and Omega2 = V2^T Omega has spectral norm 1, so
    # x = ||Omega2||^2 ||Omega1^+||^2 = 1/4.  sigma_{l-p+1} = sigma_2 = 1.
    s = np.array([2.0, 1.0, 0.5, 0.25])
    V = np.eye(4)
    om = np.array([[2.0, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, 0]])
    r3, r17, r65, r257, r1025 = (np.sqrt(v) for v in (3.0, 17.0, 65.0, 257.0, 1025.0))
    # Theorem 4: sigma_1 / sqrt(1 + x (sigma_2/sigma_1)^(4q+4))
    #   q = 0: 2 / sqrt(1 + 1/64) = 16/sqrt(65);  q = 1: 2 / sqrt(1 + 1/1024) = 64/sqrt(1025)
    assert np.isclose(bounds.thm4_lower(s, V, om, 1, 0)[0], 16 / r65, rtol=1e-14, atol=0)
    assert np.isclose(bounds.thm4_lower(s, V, om, 1, 1)[0], 64 / r1025, rtol=1e-14, atol=0)
    # Theorem 5 (sigma_k = sigma_1 = 2, sigma_{k+1} = 1):
    #   q = 0: alpha = 1/2, beta = 1/4, eta = 1, tau = 1/2
    #     sqrt(alpha^2 x / (1 + beta^2 x)) = 2/sqrt(65), sqrt(eta^2 x / (1 + tau^2 x)) = 2/sqrt(17)
    #   q = 1: (sigma_2/sigma_1)^2 = 1/4 scales alpha, beta, eta, tau:
    #     2/sqrt(1025) and 2/sqrt(257)
    #   ||A0||_2 = 1, ||A0||_F = sqrt(1 + 1/4 + 1/16) = sqrt(21)/4
    a0f = np.sqrt(21.0) / 4
    assert np.isclose(bounds.thm5_upper(s, V, om, 1, 0, "2"), 1 + 2 / r65 + 2 / r17, rtol=1e-14, atol=0)
    assert np.isclose(bounds.thm5_upper(s, V, om, 1, 0, "fro"), a0f + 2 / r65 + 2 / r17, rtol=1e-14, atol=0)
    assert np.isclose(bounds.thm5_upper(s, V, om, 1, 1, "2"), 1 + 2 / r1025 + 2 / r257, rtol=1e-14, atol=0)
    # Theorems 6 and 7: nu = nu1 nu2, nu1 = sqrt(n - l + p) + sqrt(l) + 7 = 7 + 2 sqrt(3),
    # nu2 = 4 e sqrt(l) / (p + 1) = 4 e sqrt(3) / 3; gamma_1 = sigma_2 / sigma_1 = 1/2
    nu = (7 + 2 * r3) * 4 * np.e * r3 / 3
    assert np.isclose(bounds.thm6_expected_lower(s, 4, 1, 2, 0)[0], 2 / np.sqrt(1 + nu ** 2 / 16), rtol=1e-14)
    assert np.isclose(bounds.thm6_expected_lower(s, 4, 1, 2, 1)[0], 2 / np.sqrt(1 + nu ** 2 / 256), rtol=1e-14)
    # (1 + gamma_k) sqrt(k) nu sigma_{k+1} gamma_k^(2q) = 1.5 nu (q = 0), 0.375 nu (q = 1)
    assert np.isclose(bounds.thm7_expected_upper(s, 4, 1, 2, 0, "2"), 1 + 1.5 * nu, rtol=1e-14)
    assert np.isclose(bounds.thm7_expected_upper(s, 4, 1, 2, 1, "2"), 1 + 0.375 * nu, rtol=1e-14)
    assert np.isclose(bounds.thm7_expected_upper(s, 4, 1, 2, 1, "fro"), a0f + 0.375 * nu, rtol=1e-14)


# -- planted mistakes: each plausible slip in the oracle must trip a pin above --

def test_planted_dropped_qr_column_is_caught(monkeypatch):
    A = inputs.exact_rank(120, 80, 5, seed=1)
    real = orc.householder_qr

    def bad_qr(T):
        Q, R = real(T)
        Q = Q.copy()
        Q[:, -1] = 0.0
        return Q, R
    monkeypatch.setattr(orc, "householder_qr", bad_qr)
    U, S, V = orc.sorsvd(A, 5, 0, 0, seed=0)
    assert _rel(A, U, S, V) > 1e-6          # the exact-recovery pin would fail


def test_planted_transposed_small_svd_factor_is_caught(monkeypatch):
    A = inputs.exact_rank(120, 80, 5, seed=2)
    real = orc.jacobi_svd

    def bad_svd(M):
        U, s, V, sw = real(M)
        return U, s, V.T.copy(), sw
    monkeypatch.setattr(orc, "jacobi_svd", bad_svd)
    U, S, V = orc.sorsvd(A, 5, 3, 0, seed=0)
    assert _rel(A, U, S, V) > 1e-6
