"""GPU: batched persistent recovery and the differentiable fixed-support LS step."""
import numpy as np
import pytest

import oracle
from oracle import adjoint, greedy, ls
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, dev, measurements, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def _prepare(B, probs):
    ops, ys, truths, refs = [], [], [], []
    for p in probs:
        ref_op = oracle.Operator(p.N, p.M, p.op_seed)
        s, y = measurements(p, ref_op)
        ops.append(B.Operator(p.N, p.M, p.op_seed))
        ys.append(to_dev(y))
        truths.append(s)
        refs.append(ref_op)
    return ops, ys, truths, refs


def test_batched_equals_single_bitwise(B):
    """Mixed sizes (cluster sizes 1, 2, 4) and decoders in one call equal one call per signal."""
    probs = [p for p in synth.batched_workload(B=40, seed=0x0B100, e_min=8, e_max=16) if p.K <= 400][:14]
    assert len({p.N for p in probs}) >= 4
    ops, ys, _, _ = _prepare(B, probs)
    Ks = [p.K for p in probs]
    algos = [p.algo for p in probs]
    s_b, k_b, stats = B.recover_batched(ops, ys, Ks, algos, 1e-6, 200, want_stats=True)
    assert all(st["status"] == 0 for st in stats)
    for i, (op, y, p) in enumerate(zip(ops, ys, probs)):
        s1, k1 = op.recover(y, p.K, p.algo, 1e-6, 200)
        assert torch.equal(s_b[i], s1), i
        assert torch.equal(k_b[i], k1), i


def test_batched_small_signals_match_oracle(B):
    probs = [p for p in synth.batched_workload(B=60, seed=0x0B200, e_min=8, e_max=12) if p.K <= 120][:10]
    ops, ys, truths, refs = _prepare(B, probs)
    s_b, k_b = B.recover_batched(ops, ys, [p.K for p in probs], [p.algo for p in probs], 1e-6, 200)
    for i, p in enumerate(probs):
        ref = greedy.recover(refs[i], ys[i].cpu().numpy().astype(np.float64), p.K, p.algo)
        got = s_b[i].cpu().numpy()
        if ref["near_ties"] == 0:
            assert np.array_equal(k_b[i].cpu().numpy(), ref["S"]), i
        assert rel(got, ref["s"]) <= SHAT_TOL, (i, p)


# ---------------------------------------------------------------- differentiable LS step
def _ls_setup(Bsz=4, N=1 << 16, M=1 << 14, k=1024):
    op_seed = 0x0C5005
    ref = oracle.Operator(N, M, op_seed)
    g = np.random.default_rng(3)
    S = np.sort(g.choice(N, k, replace=False)).astype(np.int32)
    s_true = g.standard_normal((Bsz, k))
    y = np.stack([ref.apply_support(S, s_true[b]) + 1e-2 * g.standard_normal(M) for b in range(Bsz)])
    return ref, op_seed, S, s_true, y.astype(np.float32)


def test_adjoint_matches_dense_pinv_gradient(B):
    ref, seed, S, s_true, y = _ls_setup()
    op = B.Operator(ref.N, ref.M, seed)
    Bsz = y.shape[0]
    Sd = to_dev(np.tile(S, (Bsz, 1)))
    yd = to_dev(y).requires_grad_(True)
    sS = B.CGLeastSquares.apply(yd, Sd, op, 1e-7, 300)
    loss = ((sS - to_dev(s_true.astype(np.float32))) ** 2).sum()
    loss.backward()
    grad = yd.grad.cpu().numpy()
    for b in range(Bsz):
        _, want = adjoint.loss_grad_y(ref, S, y[b].astype(np.float64), s_true[b])
        assert rel(grad[b], want) <= 1e-3


def test_adjoint_central_difference(B):
    """L(y) = ||s_S(y) - s_true||^2 is quadratic in y, so the central difference is exact up to
    rounding for any step; the GPU forward gives L, the GPU adjoint gives the gradient."""
    ref, seed, S, s_true, y = _ls_setup(Bsz=1)
    op = B.Operator(ref.N, ref.M, seed)
    Sd = to_dev(S[None, :])

    def L(yv):
        sS = op.ls_solve(Sd, to_dev(yv[None, :].astype(np.float32)), 1e-7, 300).cpu().numpy()[0]
        return float(((sS.astype(np.float64) - s_true[0]) ** 2).sum())

    sS = op.ls_solve(Sd, to_dev(y), 1e-7, 300)
    g = 2 * (sS - to_dev(s_true.astype(np.float32)))
    grad = op.ls_backward(Sd, g.contiguous(), 1e-7, 300).cpu().numpy()[0].astype(np.float64)
    rng = np.random.default_rng(9)
    eps = 0.05 * np.linalg.norm(y[0])
    for _ in range(3):
        v = rng.standard_normal(ref.M)
        v /= np.linalg.norm(v)
        fd = (L(y[0] + eps * v) - L(y[0] - eps * v)) / (2 * eps)
        assert abs(fd - v @ grad) <= 1e-3 * max(1.0, np.linalg.norm(grad))


def test_ls_solve_batched_full_size(B):
    ref, seed, S, s_true, y = _ls_setup(Bsz=3)
    op = B.Operator(ref.N, ref.M, seed)
    got = op.ls_solve(to_dev(np.tile(S, (3, 1))), to_dev(y), 1e-7, 300).cpu().numpy()
    for b in range(3):
        assert rel(got[b], ls.ls(ref, S, y[b].astype(np.float64))) <= SHAT_TOL
