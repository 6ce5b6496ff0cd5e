"""GPU edge cases of the public API: empty batches, K = 0 inside a batch, a support of one entry,
the smallest N, work issued on a non-default stream, and two operators used concurrently."""
import numpy as np
import pytest

import oracle
from oracle import greedy, ls
from paper_1509_03979_gb300 import synth
from tests.gpu_common import APPLY_TOL, SHAT_TOL, measurements, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def test_empty_and_zero_k_batches(B):
    s_out, supp = B.recover_batched([], [], [], [], 1e-6, 100)
    assert s_out == [] and supp == []
    N, M = 1024, 256
    ref = oracle.Operator(N, M, 2)
    op = B.Operator(N, M, 2)
    p = synth.Problem(N=N, M=M, K=20, algo="omp", op_seed=2, signal_seed=3, noise_seed=4, noise_rel=0.0)
    _, y = measurements(p, ref)
    yd = to_dev(y)
    s_b, k_b, st = B.recover_batched([op, op], [yd, yd], [0, 20], ["omp", "sp"], 1e-6, 100, want_stats=True)
    assert torch.count_nonzero(s_b[0]).item() == 0
    want = greedy.recover(ref, y.astype(np.float64), 20, "sp")
    assert rel(s_b[1].cpu().numpy(), want["s"]) <= SHAT_TOL
    assert st[1]["status"] == 0


def test_single_entry_support_and_smallest_n(B):
    N, M = 16, 8
    ref = oracle.Operator(N, M, 11)
    op = B.Operator(N, M, 11)
    x = np.random.default_rng(0).standard_normal(N).astype(np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    S = np.array([[5]], dtype=np.int32)
    y = np.random.default_rng(1).standard_normal(M).astype(np.float32)
    sS = op.ls_solve(to_dev(S), to_dev(y[None, :]), 1e-7, 50).cpu().numpy()[0]
    assert rel(sS, ls.ls(ref, S[0], y.astype(np.float64))) <= SHAT_TOL
    s_hat, supp = op.recover(to_dev(y), 1, "omp", 1e-6, 50)
    want = greedy.recover(ref, y.astype(np.float64), 1, "omp")
    assert rel(s_hat.cpu().numpy(), want["s"]) <= SHAT_TOL


def test_non_default_stream_and_two_operators_concurrently(B):
    N, M = 1 << 15, 6000
    refs = [oracle.Operator(N, M, 21), oracle.Operator(N, M, 22)]
    ops = [B.Operator(N, M, 21), B.Operator(N, M, 22)]
    g = np.random.default_rng(5)
    X = [g.standard_normal((40, N)).astype(np.float32) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for op, x, s in zip(ops, X, streams):
        with torch.cuda.stream(s):
            outs.append(op.apply_batched(to_dev(x)))
    torch.cuda.synchronize()
    for op, ref, x, y in zip(ops, refs, X, outs):
        op.sync()
        got = y.cpu().numpy()
        for b in (0, 17, 39):
            assert rel(got[b], ref.apply(x[b].astype(np.float64))) <= APPLY_TOL


@pytest.mark.parametrize("algo", ["omp", "sp", "ompr", "cosamp"])
def test_full_sampling_m_equals_n(B, algo):
    """M = N keeps every DCT row: A is orthonormal, so every decoder recovers a noiseless
    K-sparse signal exactly."""
    N = M = 1024
    K = 50
    ref = oracle.Operator(N, M, 31)
    s = synth.sparse_gaussian(N, K, 32)
    y = ref.apply(s).astype(np.float32)
    op = B.Operator(N, M, 31)
    s_hat, supp = op.recover(to_dev(y), K, algo, 1e-6, 100)
    assert op.stats()["status"] == 0
    assert np.array_equal(supp.cpu().numpy(), np.flatnonzero(s))
    assert rel(s_hat.cpu().numpy(), s) <= SHAT_TOL


def test_single_measurement(B):
    """M = 1: one DCT row; A, A^T and a one-entry OMP recovery against the oracle."""
    N, M = 64, 1
    ref = oracle.Operator(N, M, 41)
    op = B.Operator(N, M, 41)
    x = np.random.default_rng(2).standard_normal(N).astype(np.float32)
    u = np.array([0.75], dtype=np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply_t(to_dev(u)).cpu().numpy(), ref.apply_t(u.astype(np.float64))) <= APPLY_TOL
    replay_parity(op, ref, u, 1, "omp", 1e-6, 10)
