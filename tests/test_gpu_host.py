"""sorsvd_run_host (A, U, S, V in host memory) against sorsvd_run on the same
data.  The host entry point copies A in column blocks and makes the
transposed copy block by block, then queues the same kernels in the same
order, so the factors must agree bit for bit with the device entry point
(which the oracle gates in test_gpu_parity.py).  Pinned and pageable host
buffers, a host leading dimension larger than m, and every dtype family.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1804_00462_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_00462_gb300 import native
    return native


def host_colmajor(store: np.ndarray, dt: str, pinned: bool, ld: int):
    """Fortran-ordered numpy storage -> column-major CPU tensor m x n with
    leading dimension ld (rows past m hold NaN: they must never be read)."""
    m, n = store.shape
    buf = np.empty((n, ld), dtype=store.dtype)
    if dt == "bf16":
        buf.view(np.uint16)[:] = 0x7FC0            # bf16 NaN
    else:
        buf[:] = np.nan
    buf[:, :m] = store.T
    x = torch.from_numpy(buf.view(np.int16)).view(torch.bfloat16) if dt == "bf16" else torch.from_numpy(buf)
    if pinned:
        x = x.pin_memory()
    return x[:, :m].T


def device_colmajor(store: np.ndarray, dt: str):
    t = np.ascontiguousarray(store.T)
    x = torch.from_numpy(t.view(np.int16)).cuda().view(torch.bfloat16) if dt == "bf16" else torch.from_numpy(t).cuda()
    return x.T


# m * element size is a multiple of 16 bytes, so the device entry point
# (lda = m) takes the same tensor-core paths as the host one (padded ld)
@pytest.mark.parametrize("dt,m,n,k,p,q", [("f32", 2096, 1300, 30, 10, 1), ("tf32", 1504, 4100, 24, 8, 1),
                                          ("bf16", 3008, 1500, 40, 8, 1), ("f64", 400, 300, 12, 4, 1)])
@pytest.mark.parametrize("pinned", [True, False])
def test_run_host_matches_run(nat, dt, m, n, k, p, q, pinned):
    A64, _, _, _ = inputs.noisy_poly(m, n, min(m, n) // 2, 1e-3, seed=5)
    store, _ = inputs.to_storage(A64, dt)
    Ud, Sd, Vd = nat.run(device_colmajor(store, dt), k, p, q, seed=9, dtype=dt, check=True)
    Ah = host_colmajor(store, dt, pinned, m + 5)
    ws = nat.alloc_workspace(m, n, k, p, dt, nat.FLAG_HOST_IO)
    Uh, Sh, Vh = nat.run_host(Ah, k, p, q, seed=9, dtype=dt, workspace=ws)
    torch.cuda.synchronize()
    st, _ = nat.get_status(ws)
    assert st == 0
    assert not Uh.is_cuda and Uh.shape == (m, k) and Vh.shape == (n, k)
    assert torch.equal(Sh, Sd.cpu())
    assert torch.equal(Uh, Ud.cpu()) and torch.equal(Vh, Vd.cpu())


def test_run_host_workspace_and_arguments(nat):
    m, n, k, p = 500, 400, 10, 5
    base = nat.workspace_size(m, n, k, p, "f32", 0)
    host = nat.workspace_size(m, n, k, p, "f32", nat.FLAG_HOST_IO)
    # the device copies of A, U, S and V come on top
    assert host >= base + (m * n + m * k + k + n * k) * 4
    A = torch.zeros(m, n, dtype=torch.float32)
    small = nat.alloc_workspace(m, n, k, p, "f32", 0)
    with pytest.raises(nat.SorsvdError):
        nat.run_host(A, k, p, 1, dtype="f32", workspace=small)
    with pytest.raises(ValueError):
        nat.run_host(A.cuda(), k, p, 1, dtype="f32")
