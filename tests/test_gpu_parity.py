"""GPU parity: every hot-path step through the C ABI against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, greedy, ls
from paper_1509_03979_gb300 import synth
from tests.gpu_common import APPLY_TOL, SHAT_TOL, dev, measurements, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


# ------------------------------------------------------------------ operator A and A^T
SIZES = [(16, 8), (32, 32), (64, 20), (1024, 256), (4096, 1024), (1 << 14, 3000), (1 << 15, 1 << 13),
         (1 << 16, 1 << 14), (1 << 17, 40000), (1 << 18, 1 << 16)]


@pytest.mark.parametrize("N,M", SIZES)
def test_apply_and_transpose_match_oracle(B, N, M):
    seed = 1000 + N + M
    op = B.Operator(N, M, seed)
    ref = oracle.Operator(N, M, seed)
    om, d = op.export()
    assert np.array_equal(om, ref.omega) and np.array_equal(d.astype(float), ref.d)
    g = np.random.default_rng(N)
    x = g.standard_normal(N).astype(np.float32)
    u = g.standard_normal(M).astype(np.float32)
    y = op.apply(to_dev(x)).cpu().numpy()
    xt = op.apply_t(to_dev(u)).cpu().numpy()
    assert rel(y, ref.apply(x.astype(np.float64))) <= APPLY_TOL
    assert rel(xt, ref.apply_t(u.astype(np.float64))) <= APPLY_TOL


@pytest.mark.parametrize("N,M", [(256, 64), (1 << 16, 1 << 14), (1 << 18, 1 << 16)])
def test_rows_orthonormal_on_gpu(B, N, M):
    # A A^T = I_M: applying A after A^T returns the input
    op = B.Operator(N, M, 7)
    u = np.random.default_rng(1).standard_normal(M).astype(np.float32)
    back = op.apply(op.apply_t(to_dev(u))).cpu().numpy()
    assert rel(back, u) <= 2 * APPLY_TOL


def test_sparse_columns_closed_form(B):
    N, M = 4096, 512
    op = B.Operator(N, M, 3)
    ref = oracle.Operator(N, M, 3)
    for j in [0, 1, 2, 1000, N // 2, N - 1]:
        e = np.zeros(N, dtype=np.float32)
        e[j] = 1
        col = op.apply(to_dev(e)).cpu().numpy()
        assert np.abs(col - ref.columns([j])[:, 0]).max() <= 1e-6


# ------------------------------------------------------------------ fixed-support LS
@pytest.mark.parametrize("N,M,k", [(1024, 256, 30), (4096, 1024, 64), (1 << 16, 1 << 14, 1024)])
def test_ls_solve_matches_closed_form(B, N, M, k):
    op = B.Operator(N, M, 11)
    ref = oracle.Operator(N, M, 11)
    g = np.random.default_rng(k)
    S = np.sort(g.choice(N, k, replace=False)).astype(np.int32)
    y = g.standard_normal(M).astype(np.float32)
    got = op.ls_solve(to_dev(S), to_dev(y), cg_tol=1e-7, cg_maxit=200).cpu().numpy()
    want = ls.ls(ref, S, y.astype(np.float64))
    assert rel(got, want) <= SHAT_TOL


def test_ls_backward_matches_pinv(B):
    N, M, k = 4096, 1024, 64
    op = B.Operator(N, M, 12)
    ref = oracle.Operator(N, M, 12)
    g = np.random.default_rng(5)
    S = np.sort(g.choice(N, k, replace=False)).astype(np.int32)
    cot = g.standard_normal(k).astype(np.float32)
    got = op.ls_backward(to_dev(S), to_dev(cot), cg_tol=1e-7, cg_maxit=200).cpu().numpy()
    want = adjoint.ls_backward(ref, S, cot.astype(np.float64))
    assert rel(got, want) <= 1e-4


# ------------------------------------------------------------------ greedy decoders
@pytest.mark.parametrize("algo", ["omp", "sp", "ompr", "cosamp"])
def test_workload1_size_all_decoders(B, algo):
    """The N = 4096, M = 1024, K = 64 workload, selection by selection against the oracle."""
    p = synth.workload(1)
    ref_op = oracle.Operator(p.N, p.M, p.op_seed)
    s_true, y = measurements(p, ref_op)
    op = B.Operator(p.N, p.M, p.op_seed)
    rep, s, supp, st, ref = replay_parity(op, ref_op, y, p.K, algo, 1e-6, 200)
    assert np.all(np.diff(supp) > 0), "support must be sorted ascending"
    assert rep["selections"] >= (p.K if algo == "omp" else 1)


@pytest.mark.parametrize("N,M,K,algo,noise", [
    (256, 64, 8, "omp", 0.0), (2048, 512, 40, "sp", 1e-3), (1 << 14, 1 << 12, 300, "sp", 1e-3),
    (1 << 15, 1 << 13, 500, "ompr", 0.0), (1 << 16, 1 << 14, 800, "sp", 1e-3), (1 << 14, 3000, 200, "omp", 1e-3)])
def test_decoders_ragged_sizes(B, N, M, K, algo, noise):
    p = synth.Problem(N, M, K, algo, 7 * N + 1, 7 * N + 2, 7 * N + 3, noise)
    ref_op = oracle.Operator(N, M, p.op_seed)
    s_true, y = measurements(p, ref_op)
    op = B.Operator(N, M, p.op_seed)
    replay_parity(op, ref_op, y, K, algo, 1e-6, 200)


def test_k_zero_returns_zeros(B):
    op = B.Operator(1024, 256, 1)
    y = to_dev(np.ones(256, dtype=np.float32))
    s, supp = op.recover(y, 0, "omp")
    assert float(s.abs().max()) == 0.0


def test_invalid_arguments_raise(B):
    op = B.Operator(1024, 256, 1)
    y = to_dev(np.ones(256, dtype=np.float32))
    with pytest.raises(RuntimeError):
        op.recover(y, 200, "sp")          # 2K > M
    with pytest.raises(RuntimeError):
        op.recover(y, 300, "omp")         # K > M
    with pytest.raises(RuntimeError):
        B.Operator(1 << 25, 10, 1)        # N beyond the streamed path
