"""Robust PCA by inexact ALM with SOR-SVD as the low-rank step (Table 3,
"ALM-SOR-SVD", Sec. V-C), in binary64 on the CPU.

TEST INFRASTRUCTURE: only tests and the CPU baseline leg of ``bench.py`` may
import this package.

Per iteration (Table 3):
  (U, Z, V) = sorsvd(X - S_k + Y_k / mu_k)
  L_{k+1}   = U shrink_{1/mu_k}(Z) V^T
  S_{k+1}   = shrink_{lambda/mu_k}(X - L_{k+1} + Y_k / mu_k)
  Y_{k+1}   = Y_k + mu_k (X - L_{k+1} - S_{k+1})
  mu_{k+1}  = min(rho mu_k, mu_bar)
with shrink_e(x) = sgn(x) max(|x| - e, 0), stopping once
||X - L - S||_F < tol ||X||_F (Sec. V-C-1).

Readings where the paper is silent or garbled: the table prints
mu_{k+1} = max(rho mu_k, mu_bar), which would jump straight to mu_bar; it is
read as the usual cap min(rho mu_k, mu_bar).  The initial values are "those
suggested in" the cited inexact-ALM work but are not printed; the defaults
below are lambda = 1/sqrt(max(m, n)), Y_0 = X / max(||X||_2, ||X||_inf/lambda),
mu_0 = 1.25/||X||_2, rho = 1.5, mu_bar = 1e7 mu_0, S_0 = 0.  ||X||_2 is
supplied by the caller (``norm2``) so that both implementations start from
the same number.  Each inner SOR-SVD call uses seed + iteration index
("a random start").
"""
from __future__ import annotations

import math

import numpy as np

from .sor_svd import sorsvd


def shrink(x: np.ndarray, eps: float) -> np.ndarray:
    return np.sign(x) * np.maximum(np.abs(x) - eps, 0.0)


def rpca_alm(X: np.ndarray, k: int, p: int, q: int, seed: int, norm2: float, *,
             tol: float = 1e-7, max_iter: int = 50, rho: float = 1.5,
             omega_dtype: str = "f64", history: bool = False):
    X = np.asarray(X, dtype=np.float64)
    m, n = X.shape
    lam = 1.0 / math.sqrt(max(m, n))
    norm_inf = float(np.max(np.abs(X)))
    Y = X / max(norm2, norm_inf / lam)
    mu = 1.25 / norm2
    mu_bar = mu * 1e7
    S = np.zeros_like(X)
    L = np.zeros_like(X)
    nx = float(np.linalg.norm(X))
    xis = []
    it = 0
    for it in range(1, max_iter + 1):
        G = X - S + Y / mu
        U, Z, V = sorsvd(G, k, p, q, seed + it - 1, omega_dtype=omega_dtype)
        L = (U * shrink(Z, 1.0 / mu)[None, :]) @ V.T
        S = shrink(X - L + Y / mu, lam / mu)
        R = X - L - S
        Y = Y + mu * R
        mu = min(rho * mu, mu_bar)
        xi = float(np.linalg.norm(R)) / nx
        xis.append(xi)
        if xi < tol:
            break
    out = dict(L=L, S=S, iters=it, xi=xis[-1] if xis else float("nan"))
    if history:
        out["xi_history"] = xis
    return out
