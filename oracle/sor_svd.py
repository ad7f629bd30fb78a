"""SOR-SVD (subspace-orbit randomized SVD) in binary64 on the CPU.

TEST INFRASTRUCTURE: only tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.

Follows Algorithm 3 (SOR-SVD with power method, Sec. III).  The method
draws a standard Gaussian test matrix Omega (n x l, l = k + p) and builds two
sketches alternately, T1 = A T2 and then T2 = A^T T1 (eqs. T1 and AT1),
starting from T2 = Omega and going round q + 1 times (q = 0 is the basic
method of Sec. III).  QR factorisations of the final sketches give orthonormal
bases Q1 (m x l) and Q2 (n x l); the l x l core is M = Q1^T A Q2 (eq. M).  The
SVD of M, cut to its k largest singular values, gives U~_k, S~_k, V~_k, and
the rank-k factors are U = Q1 U~_k, S = S~_k, V = Q2 V~_k (A_hat = U S V^T;
the paper prints the last factor without its transpose).

``mode="literal"`` runs the alternating products exactly as printed.  ``mode="stabilised"``
replaces T2 by the Q factor of its QR decomposition before every pass i > 1.
By Gu's lemma (Sec. IV, Lemma 1: QR projectors are invariant under right
multiplication by a nonsingular matrix) this changes neither Q1 Q1^T nor
Q2 Q2^T in exact arithmetic, so A_hat is unchanged; it only keeps the
columns of T2 from collapsing onto the leading singular direction.

``core="two_pass"`` replaces the core product by the paper's M_approx =
Q1^T T1 (Q2^T T2_prev)^+ (the second core option of Algorithm 3), where T2_prev
is the T2 that entered the last pass (the "non-updated" T2, Sec. III).

``rsvd`` and ``tsrsvd`` are the paper's comparison methods on the same
steps: the randomized SVD (Algorithm 1) and the two-sided randomized SVD
(Algorithm 2).

The GEMMs are numpy matmul calls (a library primitive); QR and SVD are the
oracle's own Householder and one-sided Jacobi routines.
"""
from __future__ import annotations

import math

import numpy as np

from .linalg import householder_qr, jacobi_svd
from .philox import gaussian_matrix


def sorsvd(A: np.ndarray, k: int, p: int, q: int, seed: int, *,
           omega_dtype: str = "f64", mode: str = "stabilised",
           core: str = "three_pass", omega: np.ndarray | None = None,
           return_intermediates: bool = False):
    """Rank-k SOR-SVD of A (m x n, any m, n with l = k+p <= min(m, n)).

    ``A`` is used exactly as given (binary64).  ``omega_dtype`` rounds the
    Gaussian test matrix to the precision the GPU multiplies it in.
    Returns (U m x k, S k, V n x k) or, with ``return_intermediates``,
    (U, S, V, info dict).
    """
    A = np.asanyarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if not (1 <= k <= l <= min(m, n)):
        raise ValueError(f"need 1 <= k <= l=k+p <= min(m,n); got k={k}, p={p}, shape={A.shape}")
    if q < 0:
        raise ValueError("q must be >= 0")
    if omega is None:
        omega = gaussian_matrix(n, l, seed, 0, omega_dtype)
    T2 = np.array(omega, dtype=np.float64, copy=True)
    T2_prev = T2
    for i in range(1, q + 2):
        if i > 1 and mode == "stabilised":
            T2, _ = householder_qr(T2)
        elif mode not in ("stabilised", "literal"):
            raise ValueError(f"unknown mode {mode!r}")
        T2_prev = T2
        T1 = A @ T2
        T2 = A.T @ T1
    Q1, R1 = householder_qr(T1)
    Q2, R2 = householder_qr(T2)
    if core == "three_pass":
        M = Q1.T @ (A @ Q2)
    elif core == "two_pass":
        M = (Q1.T @ T1) @ np.linalg.pinv(Q2.T @ T2_prev)
    else:
        raise ValueError(f"unknown core {core!r}")
    Ut, st, Vt, sweeps = jacobi_svd(M)
    U = Q1 @ Ut[:, :k]
    V = Q2 @ Vt[:, :k]
    S = st[:k].copy()
    if return_intermediates:
        info = dict(omega=omega, T1=T1, T2=T2, Q1=Q1, Q2=Q2, R1=R1, R2=R2, M=M,
                    sigma_core=st, sweeps=sweeps)
        return U, S, V, info
    return U, S, V


def rsvd(A: np.ndarray, k: int, p: int, q: int, seed: int, *, omega_dtype: str = "f64",
         mode: str = "stabilised"):
    """Randomized SVD, R-SVD (Algorithm 1, Sec. II), cut to rank k.

    Omega (n x l) is the same Gaussian test matrix as SOR-SVD's;
    Y = (A A^T)^q A Omega; Y = Q R; B = Q^T A (l x n); B = U~ S W^T (SVD);
    A ~ (Q U~_k) S_k W_k^T.  ``mode="stabilised"`` replaces the running
    product by the Q factor of its QR decomposition before each multiplication
    by A^T (Lemma 1: range(Q) is unchanged in exact arithmetic).
    The SVD of the wide B is taken from the one-sided Jacobi SVD of B^T
    (n x l): B^T = W S Z^T gives B = Z S W^T.
    Returns (U m x k, S k, V n x k)."""
    A = np.asanyarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if not (1 <= k <= l <= min(m, n)) or q < 0:
        raise ValueError(f"need 1 <= k <= l=k+p <= min(m,n), q >= 0; got k={k}, p={p}, q={q}, shape={A.shape}")
    omega = gaussian_matrix(n, l, seed, 0, omega_dtype)
    Y = A @ omega
    for _ in range(q):
        if mode == "stabilised":
            Y, _ = householder_qr(Y)
        elif mode != "literal":
            raise ValueError(f"unknown mode {mode!r}")
        Y = A @ (A.T @ Y)
    Q, _ = householder_qr(Y)
    B = Q.T @ A
    W, s, Z, _ = jacobi_svd(B.T)
    return Q @ Z[:, :k], s[:k].copy(), W[:, :k]


def tsrsvd(A: np.ndarray, k: int, p: int, seed: int, *, omega_dtype: str = "f64"):
    """Two-sided randomized SVD, TSR-SVD (Algorithm 2, Sec. II), cut to rank k.

    Psi1 (n x l) is SOR-SVD's Gaussian test matrix (Philox stream 0) and Psi2
    (m x l) the same generator's stream 1; Y1 = A Psi1 and Y2 = A^T Psi2;
    Y1 = Q1 R1, Y2 = Q2 R2; B_approx = Q1^T Y1 (Q2^T Psi1)^+; its SVD
    U~ S V~^T gives A ~ (Q1 U~_k) S_k (Q2 V~_k)^T.  Returns (U, S, V)."""
    A = np.asanyarray(A, dtype=np.float64)
    m, n = A.shape
    l = k + p
    if not (1 <= k <= l <= min(m, n)):
        raise ValueError(f"need 1 <= k <= l=k+p <= min(m,n); got k={k}, p={p}, shape={A.shape}")
    psi1 = gaussian_matrix(n, l, seed, 0, omega_dtype)
    psi2 = gaussian_matrix(m, l, seed, 1, omega_dtype)
    Y1 = A @ psi1
    Y2 = A.T @ psi2
    Q1, _ = householder_qr(Y1)
    Q2, _ = householder_qr(Y2)
    Bm = (Q1.T @ Y1) @ np.linalg.pinv(Q2.T @ psi1)
    Ut, st, Vt, _ = jacobi_svd(Bm)
    return Q1 @ Ut[:, :k], st[:k].copy(), Q2 @ Vt[:, :k]


def flop_count(m: int, n: int, k: int, p: int, q: int) -> float:
    """Operation count of SOR-SVD with the power method, eq. (C_SOR-SVD+PM):
    (2q+3) l C_mult + 2 l (m+n)(l+k) + 2 l^2 (m+l), with C_mult = 2mn the flops
    of one matrix-vector product with A or A^T."""
    l = k + p
    return float((2 * q + 3) * l * 2 * m * n + 2 * l * (m + n) * (l + k) + 2 * l * l * (m + l))


def recon_error_fro(A: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray,
                    block: int = 4096) -> float:
    """||A - U diag(S) V^T||_F, accumulated over row blocks in binary64."""
    A = np.asarray(A)
    m = A.shape[0]
    US = np.asarray(U, dtype=np.float64) * np.asarray(S, dtype=np.float64)[None, :]
    Vt = np.asarray(V, dtype=np.float64).T
    acc = 0.0
    for r0 in range(0, m, block):
        D = np.asarray(A[r0:r0 + block], dtype=np.float64) - US[r0:r0 + block] @ Vt
        acc += float(np.sum(D * D))
    return math.sqrt(acc)


def eckart_young(sigma: np.ndarray, k: int):
    """Optimal rank-k errors (Theorem 1): (sigma_{k+1}, sqrt(sum_{j>k} sigma_j^2))."""
    s = np.sort(np.asarray(sigma, dtype=np.float64))[::-1]
    two = float(s[k]) if s.size > k else 0.0
    fro = float(np.sqrt(np.sum(s[k:] ** 2)))
    return two, fro


def orthonormality_defect(Q: np.ndarray) -> float:
    """||Q^T Q - I||_F."""
    Q = np.asarray(Q, dtype=np.float64)
    G = Q.T @ Q
    return float(np.linalg.norm(G - np.eye(G.shape[0])))
