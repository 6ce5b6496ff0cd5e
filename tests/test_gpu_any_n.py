"""GPU parity of the any-N path (N not a power of two, 16 <= N <= 4096): one CTA holds the
signal in natural order and computes the orthonormal DCT-II / DCT-III as chirp-z transforms
over power-of-two FFTs.  Operator, LS, adjoint and every decoder against the FP64 oracle, whose
DCT takes any N (pinned against scipy's DCT at N = 1000, 999 and 24)."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, ls
from paper_1509_03979_gb300 import synth
from tests.gpu_common import APPLY_TOL, SHAT_TOL, measurements, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


@pytest.mark.parametrize("N,M", [(24, 10), (17, 17), (999, 333), (1000, 300), (3000, 900), (4095, 1000),
                                 (3 * 1024, 700)])
def test_apply_and_transpose_any_n(B, N, M):
    op = B.Operator(N, M, 500 + N)
    ref = oracle.Operator(N, M, 500 + N)
    om, d = op.export()
    assert np.array_equal(om, ref.omega) and np.array_equal(d.astype(float), ref.d)
    g = np.random.default_rng(N)
    x = g.standard_normal(N).astype(np.float32)
    u = g.standard_normal(M).astype(np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    assert rel(op.apply_t(to_dev(u)).cpu().numpy(), ref.apply_t(u.astype(np.float64))) <= APPLY_TOL
    # rows orthonormal: A A^T = I_M
    assert rel(op.apply(op.apply_t(to_dev(u))).cpu().numpy(), u) <= 2 * APPLY_TOL
    # closed-form columns
    for j in (0, 1, N // 2, N - 1):
        e = np.zeros(N, dtype=np.float32)
        e[j] = 1
        assert np.abs(op.apply(to_dev(e)).cpu().numpy() - ref.columns([j])[:, 0]).max() <= 1e-6


@pytest.mark.parametrize("N,M,K,algo,noise", [
    (1000, 300, 20, "omp", 0.0), (999, 333, 25, "sp", 1e-3), (1000, 400, 30, "ompr", 0.0),
    (1000, 360, 30, "cosamp", 1e-3), (4095, 1200, 80, "sp", 1e-3), (3 * 1024, 900, 60, "omp", 1e-3),
    (24, 12, 2, "omp", 0.0)])
def test_decoders_any_n(B, N, M, K, algo, noise):
    p = synth.Problem(N, M, K, algo, 11 * N + 1, 11 * N + 2, 11 * N + 3, noise)
    ref_op = oracle.Operator(N, M, p.op_seed)
    _, y = measurements(p, ref_op)
    op = B.Operator(N, M, p.op_seed)
    replay_parity(op, ref_op, y, K, algo, 1e-6, 200)


def test_ls_and_adjoint_any_n(B):
    N, M, k = 1000, 300, 40
    op = B.Operator(N, M, 77)
    ref = oracle.Operator(N, M, 77)
    g = np.random.default_rng(7)
    S = np.sort(g.choice(N, k, replace=False)).astype(np.int32)
    y = g.standard_normal(M).astype(np.float32)
    got = op.ls_solve(to_dev(S), to_dev(y), 1e-7, 200).cpu().numpy()
    assert rel(got, ls.ls(ref, S, y.astype(np.float64))) <= SHAT_TOL
    cot = g.standard_normal(k).astype(np.float32)
    dy = op.ls_backward(to_dev(S), to_dev(cot), 1e-7, 200).cpu().numpy()
    assert rel(dy, adjoint.ls_backward(ref, S, cot.astype(np.float64))) <= 1e-4


def test_any_n_in_a_mixed_batch_equals_single_calls(B):
    cases = [(1000, 300, 20, "omp"), (4096, 1024, 50, "sp"), (999, 333, 25, "sp"), (3000, 900, 40, "omp")]
    ops, ys = [], []
    for i, (N, M, K, algo) in enumerate(cases):
        p = synth.Problem(N, M, K, algo, 70 + i, 80 + i, 90 + i, 1e-3)
        ref = oracle.Operator(N, M, p.op_seed)
        _, y = measurements(p, ref)
        ops.append(B.Operator(N, M, p.op_seed))
        ys.append(to_dev(y))
    s_b, k_b, st = B.recover_batched(ops, ys, [c[2] for c in cases], [c[3] for c in cases], 1e-6, 200,
                                     want_stats=True)
    assert all(x["status"] == 0 for x in st)
    for i, (op, y, c) in enumerate(zip(ops, ys, cases)):
        s1, k1 = op.recover(y, c[2], c[3], 1e-6, 200)
        assert torch.equal(s_b[i], s1) and torch.equal(k_b[i], k1), i
        s2, k2 = op.recover_noalloc(y, c[2], c[3], 1e-6, 200)
        assert torch.equal(s2, s1) and torch.equal(k2, k1), i


def test_any_n_limits(B):
    with pytest.raises(RuntimeError):
        B.Operator(4097, 100, 1)                       # beyond the any-N path
    with pytest.raises(RuntimeError):
        B.Operator(1000, 300, 1, randomizer="perm")    # signs only on the any-N path
    op = B.Operator(1000, 300, 1)
    with pytest.raises(RuntimeError):
        op.set_cluster_size(2)
