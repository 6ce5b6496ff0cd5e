"""GPU: batched A / A^T through both implementations (cluster-resident and streamed) against the
FP64 oracle, element by element on the same seeded inputs."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import APPLY_TOL, dev, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

# every row count the streamed kernel has (P = N / 16384 = 2, 4, 8, 16) and ragged M
STREAM_SIZES = [(1 << 15, 1 << 13), (1 << 16, 12345), (1 << 17, 40000), (1 << 18, 1 << 16), (1 << 18, (1 << 18) - 3)]


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def _batch(N, M, nb, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((nb, N)).astype(np.float32), g.standard_normal((nb, M)).astype(np.float32)


@pytest.mark.parametrize("impl", ["cluster", "streamed"])
@pytest.mark.parametrize("N,M", STREAM_SIZES)
def test_batched_apply_matches_oracle(B, impl, N, M):
    seed = 0x5EED + N + M
    op = B.Operator(N, M, seed)
    op.set_batched_impl(impl)
    ref = oracle.Operator(N, M, seed)
    X, U = _batch(N, M, 3, N + M)
    Y = op.apply_batched(to_dev(X)).cpu().numpy()
    XT = op.apply_t_batched(to_dev(U)).cpu().numpy()
    for b in range(X.shape[0]):
        assert rel(Y[b], ref.apply(X[b].astype(np.float64))) <= APPLY_TOL, b
        assert rel(XT[b], ref.apply_t(U[b].astype(np.float64))) <= APPLY_TOL, b


def test_streamed_elementwise_and_structure(B):
    """Per-element agreement at N = 2^18 (every output within 5e-4 of the RMS output, against
    FP32 rounding of about 1e-6 per element), basis vectors (columns of A in closed form), and
    A A^T = I_M, all through the streamed path."""
    N, M, seed = 1 << 18, 1 << 16, 0x0C5002
    op = B.Operator(N, M, seed)
    op.set_batched_impl("streamed")
    ref = oracle.Operator(N, M, seed)
    X, U = _batch(N, M, 2, 11)
    Y = op.apply_batched(to_dev(X)).cpu().numpy().astype(np.float64)
    want = ref.apply(X[0].astype(np.float64))
    assert np.max(np.abs(Y[0] - want)) <= 5e-4 * np.linalg.norm(want) / np.sqrt(M)
    e = np.zeros((2, N), dtype=np.float32)
    j = 123457
    e[0, j] = 1.0
    e[1, N - 1] = 1.0
    cols = op.apply_batched(to_dev(e)).cpu().numpy().astype(np.float64)
    assert rel(cols[0], ref.columns([j])[:, 0]) <= APPLY_TOL
    assert rel(cols[1], ref.columns([N - 1])[:, 0]) <= APPLY_TOL
    back = op.apply_batched(op.apply_t_batched(to_dev(U))).cpu().numpy()
    for b in range(2):
        assert rel(back[b], U[b]) <= 2 * APPLY_TOL


def test_streamed_persistent_loop_and_ragged_batch(B):
    """More vectors than resident CTAs (each CTA walks several), compared with the cluster path;
    B = 1 and B = 0 take their own branches."""
    N, M, seed = 1 << 16, 1 << 14, 99
    op = B.Operator(N, M, seed)
    nb = 333
    X, U = _batch(N, M, nb, 5)
    Xd, Ud = to_dev(X), to_dev(U)
    op.set_batched_impl("streamed")
    Ys, XTs = op.apply_batched(Xd), op.apply_t_batched(Ud)
    op.set_batched_impl("cluster")
    Yc, XTc = op.apply_batched(Xd), op.apply_t_batched(Ud)
    torch.cuda.synchronize()
    for b in range(nb):
        assert rel(Ys[b].cpu().numpy(), Yc[b].cpu().numpy()) <= 2 * APPLY_TOL, b
        assert rel(XTs[b].cpu().numpy(), XTc[b].cpu().numpy()) <= 2 * APPLY_TOL, b
    op.set_batched_impl("streamed")
    one = op.apply_batched(Xd[:1]).cpu().numpy()
    assert rel(one[0], Ys[0].cpu().numpy()) <= 2 * APPLY_TOL
    empty = op.apply_batched(Xd[:0])
    assert empty.shape == (0, M)


def test_streamed_rejected_outside_its_sizes(B):
    for N in (1 << 14, 1 << 19):
        op = B.Operator(N, N // 4, 3)
        with pytest.raises(RuntimeError):
            op.set_batched_impl("streamed")
        op.set_batched_impl("cluster")
        op.set_batched_impl("auto")


def test_autotuner_times_candidates_and_keeps_a_correct_path(B):
    N, M, seed = 1 << 17, 30000, 4242
    op = B.Operator(N, M, seed)
    ms = op.tune_batched(40)
    for d in ("A", "AT"):
        assert set(ms[d]) == {"cluster", "streamed x1", "streamed x2", "streamed x4"}   # P = 8: at most 4
        assert all(v > 0 for v in ms[d].values())
    ref = oracle.Operator(N, M, seed)
    X, U = _batch(N, M, 3, 77)
    Y = op.apply_batched(to_dev(X)).cpu().numpy()
    XT = op.apply_t_batched(to_dev(U)).cpu().numpy()
    for b in range(3):
        assert rel(Y[b], ref.apply(X[b].astype(np.float64))) <= APPLY_TOL
        assert rel(XT[b], ref.apply_t(U[b].astype(np.float64))) <= APPLY_TOL
    small = B.Operator(1 << 12, 1000, 1)   # below the streamed sizes: only the cluster engine
    assert set(small.tune_batched(8)["A"]) == {"cluster"}
