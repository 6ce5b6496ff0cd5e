"""GPU: CoSaMP (the SP relative that merges the 2K largest correlations and keeps the pruned
LS solution without a second solve) against the FP64 oracle on the cluster and streamed paths,
inside batched launches, without device allocation, and with the permutation randomiser."""
import numpy as np
import pytest

import oracle
from oracle import greedy
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, measurements, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("N,M,K,noise", [
    (256, 96, 8, 0.0), (4096, 1024, 60, 1e-3), (1 << 15, 1 << 13, 400, 1e-3), (1 << 16, 1 << 14, 700, 0.0),
    (1 << 18, 1 << 16, 2000, 1e-3), (1 << 19, 1 << 17, 600, 1e-3)])
def test_cosamp_matches_oracle(B, N, M, K, noise):
    p = synth.Problem(N, M, K, "cosamp", 5 * N + 1, 5 * N + 2, 5 * N + 3, noise)
    ref_op = oracle.Operator(N, M, p.op_seed)
    _, y = measurements(p, ref_op)
    op = B.Operator(N, M, p.op_seed)
    rep, s_hat, supp, st, want = replay_parity(op, ref_op, y, K, "cosamp", 1e-6, 200)
    assert np.all(np.diff(supp) > 0)
    if N <= 1 << 16:
        s2, k2 = op.recover_noalloc(to_dev(y), K, "cosamp", 1e-6, 200)
        assert rel(s2.cpu().numpy(), want["s"]) <= SHAT_TOL


def test_cosamp_in_a_mixed_batch(B):
    cases = [(4096, 1024, 50, "cosamp"), (4096, 1024, 50, "sp"), (1 << 16, 1 << 14, 500, "cosamp"),
             (1 << 13, 1 << 11, 100, "omp")]
    ops, refs, ys = [], [], []
    for i, (N, M, K, algo) in enumerate(cases):
        p = synth.Problem(N, M, K, algo, 900 + i, 910 + i, 920 + i, 1e-3)
        refs.append(oracle.Operator(N, M, p.op_seed))
        _, y = measurements(p, refs[-1])
        ys.append(y)
        ops.append(B.Operator(N, M, p.op_seed))
    s_outs, supps, st = B.recover_batched(ops, [to_dev(y) for y in ys], [c[2] for c in cases],
                                          [c[3] for c in cases], 1e-6, 200, want_stats=True)
    for i, (N, M, K, algo) in enumerate(cases):
        want = greedy.recover(refs[i], ys[i].astype(np.float64), K, algo)
        assert st[i]["status"] == 0
        assert rel(s_outs[i].cpu().numpy(), want["s"]) <= SHAT_TOL, (i, algo)


def test_cosamp_with_the_permutation_randomiser(B):
    N, M, K = 1 << 14, 1 << 12, 200
    ref_op = oracle.Operator(N, M, 0x7711, randomizer="perm")
    s = synth.sparse_gaussian(N, K, 0x7712)
    y = ref_op.apply(s).astype(np.float32)
    op = B.Operator(N, M, 0x7711, randomizer="perm")
    rep, s_hat, supp, st, want = replay_parity(op, ref_op, y, K, "cosamp", 1e-6, 200)
    assert rel(s_hat, s) <= SHAT_TOL


def test_cosamp_needs_3k_le_m(B):
    op = B.Operator(1024, 256, 1)
    y = to_dev(np.ones(256, dtype=np.float32))
    with pytest.raises(RuntimeError):
        op.recover(y, 86, "cosamp")      # 3K > M
    s, _ = op.recover(y, 85, "cosamp")
    assert op.stats()["status"] == 0
