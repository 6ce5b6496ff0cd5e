"""GPU: the cluster engine at every cluster size a size allows (CTAs per signal above the
minimum), against the FP64 oracle, and the recovery autotuner that chooses among them."""
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


CASES = [(64, 20, [1, 2, 4]), (4096, 1024, [1, 2, 4, 8, 16]), (1 << 15, 2000, [2, 4, 8, 16])]


@pytest.mark.parametrize("N,M,Ps", CASES)
def test_every_cluster_size_matches_oracle(B, N, M, Ps):
    seed = 31 * N + M
    op = B.Operator(N, M, seed)
    ref = oracle.Operator(N, M, seed)
    g = np.random.default_rng(N)
    x = g.standard_normal(N).astype(np.float32)
    u = g.standard_normal(M).astype(np.float32)
    K = max(2, M // 12)
    p = synth.Problem(N=N, M=M, K=K, algo="sp", op_seed=seed, signal_seed=seed + 1, noise_seed=seed + 2,
                      noise_rel=1e-3)
    _, y = measurements(p, ref)
    S = np.sort(g.choice(N, K, replace=False)).astype(np.int32)
    for P in Ps:
        op.set_cluster_size(P)
        assert op.cluster_size() == P
        assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL, P
        assert rel(op.apply_t(to_dev(u)).cpu().numpy(), ref.apply_t(u.astype(np.float64))) <= APPLY_TOL, P
        sS = op.ls_solve(to_dev(S[None, :]), to_dev(y[None, :]), 1e-7, 300).cpu().numpy()[0]
        assert rel(sS, ls.ls(ref, S, y.astype(np.float64))) <= SHAT_TOL, P
        for a in ("omp", "sp", "ompr"):
            replay_parity(op, ref, y, K, a, 1e-6, 200)


def test_invalid_cluster_sizes(B):
    op = B.Operator(1 << 15, 4000, 3)
    for P in (1, 3, 32):          # below the minimum of 2, not a power of two, above 16
        with pytest.raises(RuntimeError):
            op.set_cluster_size(P)
    small = B.Operator(64, 20, 3)
    with pytest.raises(RuntimeError):
        small.set_cluster_size(8)  # N < 4 P^2
    big = B.Operator(1 << 19, 1 << 17, 3)
    with pytest.raises(RuntimeError):
        big.set_cluster_size(4)   # the streamed geometry has one shape
    op.set_cluster_size(0)
    assert op.cluster_size() == 2


def test_recovery_autotuner_keeps_the_fastest_correct_shape(B):
    p = synth.workload(1)
    op = B.Operator(p.N, p.M, p.op_seed)
    ref = oracle.Operator(p.N, p.M, p.op_seed)
    ms = op.tune_recover(p.K, "omp", 1e-6, 100)
    assert set(ms) == {1, 2, 4, 8, 16} and all(v > 0 for v in ms.values())
    assert op.cluster_size() == min(ms, key=ms.get)
    _, y = measurements(p, ref)
    s_hat, supp = op.recover(to_dev(y), p.K, "omp", 1e-6, 100)
    want = greedy.recover(ref, y.astype(np.float64), p.K, "omp")
    assert np.array_equal(np.sort(supp.cpu().numpy()), want["S"])
    assert rel(s_hat.cpu().numpy(), want["s"]) <= SHAT_TOL
    assert B.Operator(1 << 19, 1 << 17, 1).tune_recover(100, "sp") == {}


def test_noalloc_at_every_cluster_size(B):
    """The fixed scratch of cs_recover_noalloc covers the largest cluster at its largest N."""
    N, M = 1 << 16, 1 << 14
    p = synth.Problem(N=N, M=M, K=200, algo="omp", op_seed=5, signal_seed=6, noise_seed=7, noise_rel=0.0)
    ref = oracle.Operator(N, M, 5)
    _, y = measurements(p, ref)
    want = greedy.recover(ref, y.astype(np.float64), 200, "omp")
    op = B.Operator(N, M, 5)
    for P in (4, 8, 16):
        op.set_cluster_size(P)
        s_hat, _ = op.recover_noalloc(to_dev(y), 200, "omp")
        assert rel(s_hat.cpu().numpy(), want["s"]) <= SHAT_TOL, P
