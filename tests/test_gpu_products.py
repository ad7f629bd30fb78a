"""Tall-skinny products of the QR step (CholeskyQR: G = T^T T, Q = T R^{-1};
Sec. III) and of the output assembly (Algorithm 3), through the C ABI
(sorsvd_gram / sorsvd_apply), element by element against the binary64
product of the same fp32 inputs.

Error bound of the split-TF32 products (l <= 288 run on the tensor cores):
each operand x = hi + lo with hi the TF32 truncation (|lo| < 2^-10 |x|) and
lo truncated again by the MMA (error < 2^-20 |x|); the product is formed as
hi*hi + hi*lo + lo*hi, so one term carries an error below 3 * 2^-20 |x y|.
The fp32 accumulator adds each MMA's contribution with a relative error of
at most 2^-23 of the running sum, whose magnitude is bounded by the sum of
|x y|; n_acc such additions per output element (three MMAs per K step of 8,
over the K steps one accumulator sees) bound that part by
n_acc * 2^-23 * sum |x y|.  The Gram's per-CTA partials are summed in
binary64 (below both).  The gate is that bound times 1.01, element-wise
against (|X|^T |X|) or (|X| |B|), computed in binary64 from the same fp32
data.  The CUDA-core kernels (l > 288) round every fma in fp32: K steps of
2^-24 each, below the same gate."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_1804_00462_gb300 import native
    return native


def _rand(rows, cols, seed, scale_cols=True):
    g = np.random.default_rng(seed)
    X = g.standard_normal((rows, cols))
    if scale_cols:
        # columns graded like a power-iterated sketch (exp(-j/64))
        X *= np.exp(-np.arange(cols) / 64.0)[None, :]
    return X.astype(np.float32)


def _gram_bound(X32, rows):
    Xa = np.abs(X32.astype(np.float64))
    S = Xa.T @ Xa
    atoms_per_cta = math.ceil(math.ceil(rows / 32) / min(math.ceil(rows / 32), 148))
    n_acc = 3 * 4 * atoms_per_cta
    return (3 * 2.0 ** -20 + n_acc * 2.0 ** -23 + rows * 2.0 ** -24) * 1.01 * S


def _apply_bound(X32, B32, K):
    S = np.abs(X32.astype(np.float64)) @ np.abs(B32.astype(np.float64))
    n_acc = 3 * 4 * math.ceil(K / 32)
    return (3 * 2.0 ** -20 + n_acc * 2.0 ** -23 + K * 2.0 ** -24) * 1.01 * S


@pytest.mark.parametrize("rows,l", [(1, 1), (31, 7), (33, 16), (1000, 110), (4133, 128), (2049, 129),
                                    (5000, 200), (3001, 256), (70001, 266), (9000, 288), (3000, 300)])
def test_gram_elementwise(nat, rows, l):
    X = _rand(rows, l, seed=rows + l)
    Xd = nat.colmajor_f32(torch.from_numpy(X).cuda())
    G, st = nat.gram(Xd)
    torch.cuda.synchronize()
    assert st == 0
    Gh = G.cpu().numpy()
    X64 = X.astype(np.float64)
    ref = X64.T @ X64
    bound = _gram_bound(X, rows)
    err = np.abs(Gh - ref)
    ratio = (err / np.maximum(bound, 1e-300)).max()
    assert ratio <= 1.0, (rows, l, ratio)
    assert np.array_equal(Gh, Gh.T)                   # both halves from one sum
    G2, _ = nat.gram(Xd)
    torch.cuda.synchronize()
    assert torch.equal(G, G2)                          # fixed summation order


def _xty_bound(X32, Y32, rows, l):
    S = np.abs(X32.astype(np.float64)).T @ np.abs(Y32.astype(np.float64))
    ntypes = max(1, (-(-l // 16) * 16 + 127) // 128)
    natoms = math.ceil(rows / 32)
    n_acc = 3 * 4 * math.ceil(natoms / min(natoms, max(1, 148 // ntypes)))
    return (3 * 2.0 ** -20 + n_acc * 2.0 ** -23 + rows * 2.0 ** -24) * 1.01 * S


@pytest.mark.parametrize("rows,l", [(1, 1), (33, 16), (1000, 110), (4133, 128), (2049, 129), (5000, 200),
                                    (3001, 256), (65537, 266), (9000, 288), (3000, 300)])
def test_cross_gram_elementwise(nat, rows, l):
    X = _rand(rows, l, seed=3 * rows + l)
    Y = _rand(rows, l, seed=5 * rows + l, scale_cols=False)
    Xd = nat.colmajor_f32(torch.from_numpy(X).cuda())
    Yd = nat.colmajor_f32(torch.from_numpy(Y).cuda(), ld=rows + 8)
    G, st = nat.gram(Xd, Yd)
    torch.cuda.synchronize()
    assert st == 0
    ref = X.astype(np.float64).T @ Y.astype(np.float64)
    ratio = (np.abs(G.cpu().numpy() - ref) / np.maximum(_xty_bound(X, Y, rows, l), 1e-300)).max()
    assert ratio <= 1.0, (rows, l, ratio)
    G2, _ = nat.gram(Xd, Yd)
    torch.cuda.synchronize()
    assert torch.equal(G, G2)


@pytest.mark.parametrize("rows,K,N,tri", [(50, 7, 7, True), (1000, 110, 110, True), (1000, 110, 100, False),
                                          (5000, 128, 128, False), (4099, 266, 266, True),
                                          (70001, 266, 266, False), (70001, 266, 256, False),
                                          (3000, 288, 288, True), (3000, 200, 300, False),
                                          (2000, 300, 300, True)])
def test_apply_elementwise(nat, rows, K, N, tri):
    X = _rand(rows, K, seed=7 * rows + K)
    g = np.random.default_rng(K + N)
    B = g.standard_normal((K, N)).astype(np.float32)
    if tri:
        B = np.triu(B)
    Xd = nat.colmajor_f32(torch.from_numpy(X).cuda())
    Y, st = nat.apply(Xd, torch.from_numpy(B).cuda(), upper_tri=tri)
    torch.cuda.synchronize()
    assert st == 0
    ref = X.astype(np.float64) @ B.astype(np.float64)
    bound = _apply_bound(X, B, K)
    err = np.abs(Y.cpu().numpy().astype(np.float64) - ref)
    ratio = (err / np.maximum(bound, 1e-300)).max()
    assert ratio <= 1.0, (rows, K, N, tri, ratio)


def test_apply_writes_only_its_rows_and_columns(nat):
    # the output of a ragged last row tile and the padded columns stay untouched
    rows, K, N = 130, 40, 24
    X = _rand(rows, K, seed=1)
    B = np.random.default_rng(2).standard_normal((K, N)).astype(np.float32)
    Xd = nat.colmajor_f32(torch.from_numpy(X).cuda())
    Y, st = nat.apply(Xd, torch.from_numpy(B).cuda())
    torch.cuda.synchronize()
    assert st == 0 and Y.shape == (rows, N)
    assert np.isfinite(Y.cpu().numpy()).all()


def test_products_reject_bad_arguments(nat):
    from paper_1804_00462_gb300.native import _lib
    import ctypes as C
    X = nat.colmajor_f32(torch.ones(64, 8, device="cuda"))
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    G = torch.empty(8, 8, dtype=torch.float64, device="cuda")
    # ldx not a multiple of 4, l = 0, a workspace that is too small
    assert _lib.sorsvd_gram(X.data_ptr(), 66, None, 0, 64, 8, G.data_ptr(), 8, ws.data_ptr(), ws.numel(), None) == 1
    assert _lib.sorsvd_gram(X.data_ptr(), 64, None, 0, 64, 0, G.data_ptr(), 8, ws.data_ptr(), ws.numel(), None) == 1
    assert _lib.sorsvd_gram(X.data_ptr(), 64, X.data_ptr(), 62, 64, 8, G.data_ptr(), 8, ws.data_ptr(), ws.numel(),
                            None) == 1
    assert _lib.sorsvd_gram(X.data_ptr(), 64, None, 0, 64, 8, G.data_ptr(), 8, ws.data_ptr(), 16, None) == 7
    assert int(_lib.sorsvd_products_workspace_size(64, 0)) == 0
    assert C.sizeof(C.c_void_p) == 8
