"""Seeded synthetic inputs shaped like the paper's workloads.

This module builds test matrices only; it contains none of SOR-SVD's
arithmetic, and both the CUDA path and the CPU oracle consume what it makes.

Matrices are A = U diag(sigma) V^T with Haar-distributed U, V (the Q factor
of a Gaussian matrix with its columns multiplied by sign(R_jj), Mezzadri 2007),
as in Sec. V-A ("U and V are random orthonormal matrices"), plus the noisy and
low-rank-plus-sparse variants of the experiments.  Gaussian draws come from
numpy's Philox-based Generator seeded with ``seed`` (numpy path) or from a
seeded torch generator on the GPU (``*_torch`` builders, used where the
matrix is too large to build on the host quickly).

Storage helpers return column-major data, the layout of the C ABI.
"""
from __future__ import annotations

import math

import numpy as np

DTYPES = ("f64", "f32", "tf32", "bf16", "f16")


def rng(seed: int, stream: int = 1) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def haar(rows: int, cols: int, g: np.random.Generator) -> np.ndarray:
    Z = g.standard_normal((rows, cols))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def spectral(m: int, n: int, sigma: np.ndarray, seed: int):
    """A = U diag(sigma) V^T with Haar U (m x r), V (n x r), r = len(sigma).

    Returns (A f64 (m, n), sigma, U, V).
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.size
    g = rng(seed, 1)
    U = haar(m, r, g)
    V = haar(n, r, g)
    A = (U * sigma[None, :]) @ V.T
    return A, sigma, U, V


def sigma_cfg1(n: int = 1000, k0: int = 20) -> np.ndarray:
    """sigma_i = 1 for i <= 20, then 10^{-(i-20)/10}."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.where(i <= k0, 1.0, 10.0 ** (-(i - k0) / 10.0))


def sigma_poly(n: int, power: float = 1.0) -> np.ndarray:
    """sigma_i = i^{-power} (power 1: the paper's rapidly decaying matrix)."""
    return np.arange(1, n + 1, dtype=np.float64) ** (-power)


def sigma_exp(r: int, scale: float = 64.0) -> np.ndarray:
    """sigma_i = exp(-i/scale), i = 1..r."""
    return np.exp(-np.arange(1, r + 1, dtype=np.float64) / scale)


def cfg1(seed: int = 0, n: int = 1000):
    """FP64 square n x n, spectrum of ``sigma_cfg1``."""
    return spectral(n, n, sigma_cfg1(n), seed)


def noisy_poly(m: int, n: int, width: int, noise: float, seed: int):
    """U diag(1/i) V^T (Haar factors of ``width`` columns) + noise * N(0,1)."""
    A, s, U, V = spectral(m, n, sigma_poly(width), seed)
    A += noise * rng(seed, 2).standard_normal((m, n))
    return A, s, U, V


def cfg2(seed: int = 0, m: int = 20000, n: int = 10000, width: int = 500, noise: float = 1e-3):
    return noisy_poly(m, n, width, noise, seed)


def cfg3(seed: int = 0, m: int = 65536, n: int = 16384, width: int = 1024):
    return spectral(m, n, sigma_exp(width), seed)


def exact_rank(m: int, n: int, r: int, seed: int):
    """Rank-r matrix G H^T with Gaussian factors."""
    g = rng(seed, 3)
    return g.standard_normal((m, r)) @ g.standard_normal((n, r)).T


def batched_sizes(count: int = 512, seed: int = 0, m_range=(256, 4096), n_range=(128, 2048),
                  k_range=(8, 64)):
    """(m, n, k) per problem: m, n log-uniform, k uniform on the integers."""
    g = rng(seed, 4)
    m = np.floor(np.exp(g.uniform(math.log(m_range[0]), math.log(m_range[1]), count))).astype(int)
    n = np.floor(np.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]), count))).astype(int)
    k = g.integers(k_range[0], k_range[1] + 1, count)
    return [(int(a), int(b), int(c)) for a, b, c in zip(m, n, k)]


def batched_matrix(m: int, n: int, seed: int):
    """sigma_i = i^-2 over min(m, n), Haar factors."""
    return spectral(m, n, sigma_poly(min(m, n), 2.0), seed)


def batched_matrix_torch(m: int, n: int, seed: int, width: int | None = None, device="cuda", dtype=None):
    """sigma_i = i^-2 for i <= min(m, n) (``width`` caps the rank, default
    none) with Haar factors drawn on the device: Q of a seeded Gaussian matrix
    times sign(diag R), after Mezzadri, in binary64.  Returns a column-major
    tensor."""
    import torch
    r = min(m, n) if width is None else min(m, n, width)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))

    def haar_dev(rows):
        G = torch.randn(rows, r, generator=gen, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(G)
        return Q * torch.sign(torch.diagonal(R))[None, :]
    U = haar_dev(m)
    V = haar_dev(n)
    s = torch.from_numpy(sigma_poly(r, 2.0)).to(device)
    A = (V * s[None, :]) @ U.T                       # (n, m) row-major = A column-major
    return A.to(dtype or torch.float64).T


def rpca_problem(m: int = 25344, n: int = 400, rank: int = 5, density: float = 0.05,
                 lo: float = 1.0, hi: float = 10.0, seed: int = 0):
    """X = L + S: L = G H^T (Gaussian factors), S with Bernoulli(density)
    support and values of random sign and magnitude uniform in [lo, hi]."""
    g = rng(seed, 5)
    L = g.standard_normal((m, rank)) @ g.standard_normal((n, rank)).T
    support = g.random((m, n)) < density
    mag = g.uniform(lo, hi, (m, n))
    sgn = np.where(g.random((m, n)) < 0.5, -1.0, 1.0)
    S = np.where(support, sgn * mag, 0.0)
    return L + S, L, S


# ----------------------------------------------------------------------------
# storage
# ----------------------------------------------------------------------------

def _bf16_bits(a32: np.ndarray) -> np.ndarray:
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return b.astype(np.uint16)


def to_storage(A: np.ndarray, dtype: str):
    """Round a binary64 matrix to ``dtype`` storage.

    Returns (store, exact): ``store`` is a Fortran-ordered array holding the
    stored values (uint16 bit patterns for bf16), ``exact`` the same values as
    binary64 (what the oracle consumes).
    """
    A = np.asarray(A, dtype=np.float64)
    if dtype == "f64":
        st = np.asfortranarray(A)
        return st, st
    a32 = np.asfortranarray(A.astype(np.float32))
    if dtype in ("f32", "tf32"):
        return a32, a32.astype(np.float64)
    if dtype == "f16":
        h = np.asfortranarray(a32.astype(np.float16))
        return h, h.astype(np.float64)
    if dtype == "bf16":
        bits = np.asfortranarray(_bf16_bits(np.ascontiguousarray(a32)).reshape(A.shape))
        exact = (bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
        return bits, exact
    raise ValueError(dtype)


# ----------------------------------------------------------------------------
# large builders on the GPU (torch), for full-size runs
# ----------------------------------------------------------------------------

def spectral_torch(m: int, n: int, sigma: np.ndarray, seed: int, device="cuda",
                   noise: float = 0.0, out_dtype=None, chunk: int = 8192):
    """Column-major A = U diag(sigma) V^T (+ noise), product formed on the GPU.

    The Haar factors U (m x r), V (n x r) come from ``haar`` on the host
    (numpy); the product and the noise are formed on the GPU in fp32.
    Returns a torch tensor ``At`` of shape (n, m), contiguous: the column-major
    storage of A with lda = m, in ``out_dtype`` (default fp32).
    """
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    r = len(sigma)
    g = rng(seed, 1)
    U = torch.from_numpy(haar(m, r, g).astype(np.float32)).to(device)
    V = torch.from_numpy(haar(n, r, g).astype(np.float32)).to(device)
    Vs = V * torch.as_tensor(np.asarray(sigma, np.float32), device=device)[None, :]
    out_dtype = out_dtype or torch.float32
    At = torch.empty(n, m, device=device, dtype=out_dtype)
    for c0 in range(0, n, chunk):
        blk = Vs[c0:c0 + chunk] @ U.T
        if noise:
            blk += noise * torch.randn(blk.shape, generator=gen, device=device, dtype=torch.float32)
        At[c0:c0 + chunk] = blk.to(out_dtype)
    return At
