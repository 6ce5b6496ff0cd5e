"""GPU parity of operators with a sparsifying basis Psi = C_N^T (Sec. III-A: y = Phi Psi s; the
image experiment of Sec. IV-A takes a DCT basis): A = P_Omega C_N diag(d) C_N^T, the unknown s
the DCT coefficients of the signal.  Operator, LS, adjoint and the decoders against the FP64
oracle's Operator(..., psi="dct"), which is pinned (with no randomiser it reduces to row
sampling; a planted transposed Psi is caught)."""
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


@pytest.mark.parametrize("N,M", [(1024, 256), (1000, 300), (4096, 1024), (2049, 500), (16, 8)])
def test_basis_apply_and_transpose(B, N, M):
    op = B.Operator(N, M, 900 + N, psi="dct")
    ref = oracle.Operator(N, M, 900 + N, psi="dct")
    g = np.random.default_rng(N)
    x = g.standard_normal(N).astype(np.float32)
    u = g.standard_normal(M).astype(np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply_t(to_dev(u)).cpu().numpy(), ref.apply_t(u.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply(op.apply_t(to_dev(u))).cpu().numpy(), u) <= 2 * APPLY_TOL


def _dct_sparse_problem(N, M, K, seed, noise):
    ref = oracle.Operator(N, M, seed, psi="dct")
    s = synth.sparse_gaussian(N, K, seed + 1)          # K-sparse DCT coefficients
    y = ref.apply(s)
    if noise:
        y = y + noise * np.linalg.norm(y) / np.sqrt(M) * synth.normals(seed + 2, M)
    return ref, s, y.astype(np.float32)


@pytest.mark.parametrize("N,M,K,algo", [(1024, 300, 20, "omp"), (1000, 320, 25, "sp"), (4096, 1024, 60, "sp"),
                                        (2048, 600, 40, "cosamp"), (1000, 360, 24, "ompr")])
def test_basis_decoders_recover_dct_sparse_signals(B, N, M, K, algo):
    ref, s, y = _dct_sparse_problem(N, M, K, 40 + N + K, 0.0)
    op = B.Operator(N, M, 40 + N + K, psi="dct")
    rep, s_hat, supp, st, want = replay_parity(op, ref, y, K, algo, 1e-6, 200)
    assert rel(s_hat, s) <= SHAT_TOL                    # noiseless: the coefficients themselves
    assert np.array_equal(np.sort(supp), np.flatnonzero(s))


def test_basis_noisy_sp_and_ls_adjoint(B):
    N, M, K = 4096, 1200, 80
    ref, s, y = _dct_sparse_problem(N, M, K, 61, 1e-3)
    op = B.Operator(N, M, 61, psi="dct")
    replay_parity(op, ref, y, K, "sp", 1e-6, 200)
    S = np.sort(np.random.default_rng(2).choice(N, 50, replace=False)).astype(np.int32)
    got = op.ls_solve(to_dev(S), to_dev(y), 1e-7, 200).cpu().numpy()
    assert rel(got, ls.ls(ref, S, y.astype(np.float64))) <= SHAT_TOL
    cot = np.random.default_rng(3).standard_normal(50).astype(np.float32)
    dy = op.ls_backward(to_dev(S), to_dev(cot), 1e-7, 200).cpu().numpy()
    assert rel(dy, adjoint.ls_backward(ref, S, cot.astype(np.float64))) <= 1e-4


def test_basis_limits(B):
    with pytest.raises(RuntimeError):
        B.Operator(8192, 1000, 1, psi="dct")          # the basis runs on the any-N path, N <= 4096
    with pytest.raises(ValueError):
        B.Operator(1024, 256, 1, randomizer="perm", psi="dct")


@pytest.mark.parametrize("n1,n2,M", [(32, 64, 600), (64, 64, 1200), (30, 33, 330)])
def test_basis_2d_apply_and_transpose(B, n1, n2, M):
    N = n1 * n2
    op = B.Operator(N, M, 300 + N, psi=("dct2d", n1, n2))
    ref = oracle.Operator(N, M, 300 + N, psi=("dct2d", n1, n2))
    g = np.random.default_rng(n1 + n2)
    x = g.standard_normal(N).astype(np.float32)
    u = g.standard_normal(M).astype(np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply_t(to_dev(u)).cpu().numpy(), ref.apply_t(u.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply(op.apply_t(to_dev(u))).cpu().numpy(), u) <= 2 * APPLY_TOL


@pytest.mark.parametrize("algo", ["omp", "sp", "cosamp"])
def test_basis_2d_recovers_a_dct_sparse_image(B, algo):
    """A 64 x 64 image that is K-sparse in the separable 2-D DCT basis (the image model of the
    paper's Sec. IV-A experiment, at the size this path holds), recovered exactly from M = N/4
    measurements, selection by selection against the oracle."""
    n1 = n2 = 64
    N, M, K = n1 * n2, 1024, 40
    ref = oracle.Operator(N, M, 4242, psi=("dct2d", n1, n2))
    S = synth.sparse_gaussian(N, K, 4243)
    y = ref.apply(S).astype(np.float32)
    op = B.Operator(N, M, 4242, psi=("dct2d", n1, n2))
    rep, s_hat, supp, st, want = replay_parity(op, ref, y, K, algo, 1e-6, 200)
    assert rel(s_hat, S) <= SHAT_TOL
    image = ref._psi(s_hat.astype(np.float64))            # back to pixels
    assert rel(image, ref._psi(S)) <= SHAT_TOL
