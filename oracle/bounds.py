"""The paper's bounds on SOR-SVD, evaluated for a matrix with known SVD.

TEST INFRASTRUCTURE: only tests may import this package.

Notation (Sec. IV): A = U Sigma V^T, l = k + p; the analysis splits V into
V1 (first l - p_a columns) and V2 (the rest) and defines Omega1 = V1^T Omega,
Omega2 = V2^T Omega (eq. Omegas).  With the oversampling p = l - k used
throughout this project, the analysis parameter p_a is taken as p, so
l - p_a = k and sigma_{l-p_a+1} = sigma_{k+1}.

* ``thm4_lower``  Theorem 4 (deterministic lower bound, with the power-method
  exponent 4q + 4).  The theorem states it for sigma_j(A_hat), but its proof
  (Lemma "sv_1st") takes (Sigma_1 0 0) V^T Q~_1 as a submatrix of
  Q1 Q1^T A Q2 Q2^T, which drops the left projector Q1 Q1^T; what the proof
  establishes is the bound for sigma_j(A Q2 Q2^T).  Evaluated that way it holds
  to rounding on every draw tried, while for sigma_j(A_hat) itself it fails on
  the noisy low-rank matrix of Sec. V-A-1 at q = 0 (ratio ~0.58).
* ``thm5_upper``  Theorem 5 (deterministic error bound, 2- and F-norm).  For
  q > 0 the paper prints tau = beta / sigma_{l-p+1}; that expression does not
  reduce to the q = 0 value tau = sigma_{l-p+1}/sigma_1 and is not
  dimensionless, so it is read as tau = (sigma_k / sigma_{l-p+1}) beta, which
  does (the same relation the paper gives between eta and alpha).
* ``thm6_expected_lower`` / ``thm7_expected_upper``  Theorems 6 and 7
  (average-case bounds with nu = nu1 nu2, nu1 = sqrt(n-l+p) + sqrt(l) + 7,
  nu2 = 4 e sqrt(l) / (p+1)).
"""
from __future__ import annotations

import math

import numpy as np


def _omega_parts(V: np.ndarray, omega: np.ndarray, k: int):
    O1 = V[:, :k].T @ omega
    O2 = V[:, k:].T @ omega
    n2 = np.linalg.norm(O2, 2) if O2.size else 0.0
    smin = np.linalg.svd(O1, compute_uv=False)[-1]
    return float(n2), float(1.0 / smin)


def thm4_lower(sigma, V, omega, k, q):
    """Lower bounds on sigma_j(A_hat), j = 1..k (Theorem 4)."""
    s = np.asarray(sigma, dtype=np.float64)
    n2, inv1 = _omega_parts(V, omega, k)
    x = (n2 * inv1) ** 2
    sl = s[k]
    return s[:k] / np.sqrt(1.0 + x * (sl / s[:k]) ** (4 * q + 4))


def thm5_upper(sigma, V, omega, k, q, norm="fro"):
    """Upper bound on ||A - A_hat||_rho, rho in {"2", "fro"} (Theorem 5)."""
    s = np.asarray(sigma, dtype=np.float64)
    n2, inv1 = _omega_parts(V, omega, k)
    x = (n2 * inv1) ** 2
    s1, sk, sl = s[0], s[k - 1], s[k]
    g = (sl / sk) ** (2 * q)
    alpha = math.sqrt(k) * sl * sl / sk * g
    beta = sl * sl / (s1 * sk) * g
    eta = (sk / sl) * alpha
    tau = (sk / sl) * beta
    a0 = float(s[k]) if norm == "2" else float(np.sqrt(np.sum(s[k:] ** 2)))
    return a0 + math.sqrt(alpha ** 2 * x / (1.0 + beta ** 2 * x)) \
              + math.sqrt(eta ** 2 * x / (1.0 + tau ** 2 * x))


def _nu(n, k, p):
    l = k + p
    nu1 = math.sqrt(n - l + p) + math.sqrt(l) + 7.0
    nu2 = 4.0 * math.e * math.sqrt(l) / (p + 1)
    return nu1 * nu2


def thm6_expected_lower(sigma, n, k, p, q):
    """Lower bounds on E sigma_j(A_hat), j = 1..k (Theorem 6)."""
    s = np.asarray(sigma, dtype=np.float64)
    nu = _nu(n, k, p)
    gam = s[k] / s[:k]
    return s[:k] / np.sqrt(1.0 + nu ** 2 * gam ** (4 * q + 4))


def thm7_expected_upper(sigma, n, k, p, q, norm="fro"):
    """Upper bound on E ||A - A_hat||_rho (Theorem 7)."""
    s = np.asarray(sigma, dtype=np.float64)
    nu = _nu(n, k, p)
    gk = s[k] / s[k - 1]
    a0 = float(s[k]) if norm == "2" else float(np.sqrt(np.sum(s[k:] ** 2)))
    return a0 + (1.0 + gk) * math.sqrt(k) * nu * s[k] * gk ** (2 * q)
