"""GPU: the operator with the paper's permutation randomiser (A = P_Omega C_N Pi, Sec. III-A)
through every entry point, against the FP64 oracle built with the same permutation."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, greedy, ls
from paper_1509_03979_gb300 import synth
from tests.gpu_common import APPLY_TOL, SHAT_TOL, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("N,M", [(64, 20), (4096, 1000), (1 << 15, 9000), (1 << 18, 1 << 16), (1 << 19, 100000)])
def test_perm_apply_matches_oracle(B, N, M):
    seed = 0x9E37 + N
    op = B.Operator(N, M, seed, randomizer="perm")
    ref = oracle.Operator(N, M, seed, randomizer="perm")
    assert np.array_equal(op.export_perm().astype(np.int64), ref.perm)
    om, d = op.export()
    assert np.array_equal(om, ref.omega) and np.all(d == 1)
    g = np.random.default_rng(N)
    X = g.standard_normal((2, N)).astype(np.float32)
    U = g.standard_normal((2, M)).astype(np.float32)
    Y = op.apply_batched(to_dev(X)).cpu().numpy()
    XT = op.apply_t_batched(to_dev(U)).cpu().numpy()
    for b in range(2):
        assert rel(Y[b], ref.apply(X[b].astype(np.float64))) <= APPLY_TOL
        assert rel(XT[b], ref.apply_t(U[b].astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply(to_dev(X[0])).cpu().numpy(), ref.apply(X[0].astype(np.float64))) <= APPLY_TOL


@pytest.mark.parametrize("N,M,K", [(4096, 1024, 64), (1 << 15, 3000, 200)])
@pytest.mark.parametrize("algo", ["omp", "sp", "ompr"])
def test_perm_decoders_match_oracle(B, N, M, K, algo):
    seed = 0x51 + N + K
    ref = oracle.Operator(N, M, seed, randomizer="perm")
    s = synth.sparse_gaussian(N, K, seed + 1)
    y = ref.apply(s)
    y = (y + 1e-3 * np.linalg.norm(y) / np.sqrt(M) * synth.normals(seed + 2, M)).astype(np.float32)
    op = B.Operator(N, M, seed, randomizer="perm")
    rep, s_hat, supp, st, want = replay_parity(op, ref, y, K, algo, 1e-6, 200)
    if N <= 1 << 16:
        s2, _ = op.recover_noalloc(to_dev(y), K, algo, 1e-6, 200)
        assert rel(s2.cpu().numpy(), want["s"]) <= SHAT_TOL


def test_perm_ls_and_adjoint(B):
    N, M, k = 1 << 14, 4096, 300
    ref = oracle.Operator(N, M, 3, randomizer="perm")
    op = B.Operator(N, M, 3, randomizer="perm")
    g = np.random.default_rng(4)
    S = np.sort(g.choice(N, k, replace=False)).astype(np.int32)
    y = g.standard_normal(M).astype(np.float32)
    gr = g.standard_normal(k)
    sS = op.ls_solve(to_dev(S[None, :]), to_dev(y[None, :]), 1e-7, 300).cpu().numpy()[0]
    assert rel(sS, ls.ls(ref, S, y.astype(np.float64))) <= SHAT_TOL
    dy = op.ls_backward(to_dev(S[None, :]), to_dev(gr[None, :].astype(np.float32)), 1e-7, 300).cpu().numpy()[0]
    assert rel(dy, adjoint.ls_backward(ref, S, gr)) <= 1e-3


def test_unknown_randomizer_rejected(B):
    from paper_1509_03979_gb300 import binding
    assert not binding.lib().cs_op_create_ex(1024, 256, 1, 7)
    op = B.Operator(1024, 256, 1)
    with pytest.raises(RuntimeError):
        op.export_perm()
