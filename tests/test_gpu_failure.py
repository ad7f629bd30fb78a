"""Device-side failure paths, made to happen without faulting or hanging a
GPU: a Jacobi sweep cap of one sweep gives SORSVD_ERR_NOT_CONVERGED, and a
wait limit of 64 cycles in the tensor-core passes gives
SORSVD_ERR_TIMEOUT.  Each call returns cleanly and the next call with the
default limits is clean and matches the oracle (the aborted passes let
their copies and MMAs land and freed their tensor memory, or the next pass
could not allocate it)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1804_00462_gb300 import inputs  # noqa: E402

NOT_CONVERGED, TIMEOUT = 4, 6


@pytest.fixture(scope="module")
def nat():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_00462_gb300 import native
    yield native
    native.set_limits(0, 0)


def _problem(m, n, dt, seed):
    A64, s, _, _ = inputs.spectral(m, n, inputs.sigma_exp(min(m, n), 40.0), seed=seed)
    store, exact = inputs.to_storage(A64, dt)
    t = np.ascontiguousarray(store.T)
    if dt == "bf16":
        A = torch.from_numpy(t.view(np.int16)).cuda().view(torch.bfloat16).T
    else:
        A = torch.from_numpy(t).cuda().T
    return A, exact


def _call(nat, A, k, p, q, dt):
    ws = nat.alloc_workspace(A.shape[0], A.shape[1], k, p, dt)
    U, S, V = nat.run(A, k, p, q, seed=3, dtype=dt, workspace=ws)
    st, info = nat.get_status(ws)
    return (U, S, V), st, info


def _matches_oracle(got, exact, k, p, q, dt, tol):
    Uo, So, Vo = oracle.sorsvd(exact, k, p, q, 3, omega_dtype=dt)
    to = lambda t: t.double().cpu().numpy()
    U, S, V = got
    nA = np.linalg.norm(exact)
    r = oracle.recon_error_fro(exact, to(U), to(S), to(V)) / nA
    ro = oracle.recon_error_fro(exact, Uo, So, Vo) / nA
    return abs(r - ro) <= tol


@pytest.mark.parametrize("m,n,k,p", [(600, 400, 12, 6), (1200, 700, 60, 10)])
def test_sweep_cap_reports_not_converged(nat, m, n, k, p):
    # l = 18: one-block sweeps; l = 70: sweeps on a thread-block cluster
    A, exact = _problem(m, n, "f32", seed=m)
    before, st, _ = _call(nat, A, k, p, 1, "f32")
    assert st == 0 and _matches_oracle(before, exact, k, p, 1, "f32", 1e-5)
    nat.set_limits(0, 1)
    try:
        _, st, info = _call(nat, A, k, p, 1, "f32")
    finally:
        nat.set_limits(0, 0)
    assert st == NOT_CONVERGED, nat.status_string(st)
    assert (info >> 8) & 0xFF == 1                         # one sweep was run
    # the next call is clean and bit-identical to the one before the failure
    after, st, _ = _call(nat, A, k, p, 1, "f32")
    assert st == 0
    assert all(torch.equal(x, y) for x, y in zip(before, after))


@pytest.mark.parametrize("dt", ["bf16", "f32"])
def test_pass_wait_limit_times_out_cleanly(nat, dt):
    # 2048 x 1024 with 16-byte aligned columns: every pass runs on the
    # tensor cores (bf16 passes, F32 TF32 and split-TF32 passes)
    m, n, k, p = 2048, 1024, 24, 8
    A, exact = _problem(m, n, dt, seed=7)
    before, st, _ = _call(nat, A, k, p, 1, dt)
    assert st == 0 and _matches_oracle(before, exact, k, p, 1, dt, 1e-5 if dt == "f32" else 1e-2)
    nat.set_limits(64, 0)
    try:
        _, st, _ = _call(nat, A, k, p, 1, dt)
    finally:
        nat.set_limits(0, 0)
    assert st == TIMEOUT, nat.status_string(st)
    torch.cuda.synchronize()
    # the aborted passes freed their tensor memory and left no copy or MMA
    # behind: the next call runs cleanly, bit-identical to the one before
    after, st, _ = _call(nat, A, k, p, 1, dt)
    assert st == 0
    assert all(torch.equal(x, y) for x, y in zip(before, after))
