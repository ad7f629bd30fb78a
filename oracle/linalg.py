"""Dense building blocks of the oracle, in binary64 on the CPU.

TEST INFRASTRUCTURE: only tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.

* ``householder_qr``: thin QR by Householder reflections (the QR the method
  calls for in Algorithms 1-3, Sec. III), normalised so that diag(R) >= 0.
* ``jacobi_svd``: one-sided (Hestenes) Jacobi SVD, used for the "rank-k
  truncated SVD" of the small core matrix (Algorithm 3).  Pairs of columns are
  visited in the round-robin (tournament) order, which rotates floor(n/2)
  disjoint pairs per round; a rotation is applied whenever the cosine between
  the two columns exceeds ``tol``.
"""
from __future__ import annotations

import numpy as np

EPS64 = np.finfo(np.float64).eps


def householder_qr(T: np.ndarray):
    """Thin QR of an (m x l) matrix, m >= l, with R_jj >= 0.

    Returns (Q, R): Q is m x l with orthonormal columns, R is l x l upper
    triangular.  A zero column leaves the reflector out (R_jj = 0) and the
    matching column of Q is the reflected unit vector, so Q stays orthonormal
    for rank-deficient input.
    """
    W = np.array(T, dtype=np.float64, copy=True)
    m, l = W.shape
    if m < l:
        raise ValueError("householder_qr needs m >= l")
    vs = []
    for j in range(l):
        x = W[j:, j]
        nx = np.linalg.norm(x)
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv == 0.0:
            vs.append(None)
            continue
        v /= nv
        W[j:, j:] -= 2.0 * np.outer(v, v @ W[j:, j:])
        vs.append(v)
    R = np.triu(W[:l, :l])
    # Q = H_0 H_1 ... H_{l-1} [I_l; 0], applied from the last reflector back.
    Q = np.zeros((m, l))
    Q[np.arange(l), np.arange(l)] = 1.0
    for j in reversed(range(l)):
        v = vs[j]
        if v is None:
            continue
        Q[j:, :] -= 2.0 * np.outer(v, v @ Q[j:, :])
    sgn = np.where(np.diag(R) < 0, -1.0, 1.0)
    Q = Q * sgn[None, :]
    R = R * sgn[:, None]
    return Q, R


def _tournament_rounds(n: int):
    """Round-robin schedule of all pairs of {0..n-1} (n even: n-1 rounds)."""
    players = list(range(n)) + ([-1] if n % 2 else [])
    N = len(players)
    rounds = []
    for _ in range(N - 1):
        pairs = []
        for i in range(N // 2):
            a, b = players[i], players[N - 1 - i]
            if a >= 0 and b >= 0:
                pairs.append((min(a, b), max(a, b)))
        rounds.append(pairs)
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_svd(M: np.ndarray, tol: float | None = None, max_sweeps: int = 60):
    """One-sided Jacobi SVD of an (r x c) matrix, r >= c.

    Returns (U, s, V, sweeps) with M = U diag(s) V^T, s descending,
    U r x c, V c x c.  Sign convention: the entry of largest magnitude in each
    column of U is positive (the matching column of V flips with it).
    Columns of U for zero singular values are left as zero vectors.
    """
    W = np.array(M, dtype=np.float64, copy=True)
    r, c = W.shape
    if r < c:
        raise ValueError("jacobi_svd needs rows >= cols")
    V = np.eye(c)
    if tol is None:
        tol = max(c, 1) * EPS64
    rounds = _tournament_rounds(c)
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for pairs in rounds:
            if not pairs:
                continue
            p = np.array([a for a, _ in pairs])
            q = np.array([b for _, b in pairs])
            wp, wq = W[:, p], W[:, q]
            alpha = np.einsum("ij,ij->j", wp, wp)
            beta = np.einsum("ij,ij->j", wq, wq)
            gamma = np.einsum("ij,ij->j", wp, wq)
            act = np.abs(gamma) > tol * np.sqrt(alpha * beta)
            if not np.any(act):
                continue
            rotated = True
            p, q = p[act], q[act]
            alpha, beta, gamma = alpha[act], beta[act], gamma[act]
            zeta = (beta - alpha) / (2.0 * gamma)
            t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            cs = 1.0 / np.sqrt(1.0 + t * t)
            sn = cs * t
            wp, wq = W[:, p], W[:, q]
            W[:, p] = cs * wp - sn * wq
            W[:, q] = sn * wp + cs * wq
            vp, vq = V[:, p], V[:, q]
            V[:, p] = cs * vp - sn * vq
            V[:, q] = sn * vp + cs * vq
        if not rotated:
            break
    s = np.linalg.norm(W, axis=0)
    order = np.argsort(-s, kind="stable")
    s, W, V = s[order], W[:, order], V[:, order]
    U = np.zeros_like(W)
    nz = s > 0
    U[:, nz] = W[:, nz] / s[nz]
    idx = np.argmax(np.abs(U), axis=0)
    sgn = np.where(U[idx, np.arange(c)] < 0, -1.0, 1.0)
    U = U * sgn
    V = V * sgn
    return U, s, V, sweeps
