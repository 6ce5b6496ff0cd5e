"""GPU: library calls captured into a CUDA graph and replayed give the same results as the same
calls made directly -- single-signal recovery and apply (cluster engine), the batched operator
(both implementations), a batched recovery over two cluster sizes, a batched LS solve, and the
cooperative grid path (N = 2^19).  Every launch carries its task tables in its own parameters,
so the replays read no host memory of the capturing call."""
import numpy as np
import pytest

import oracle
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, measurements, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def capture_and_replay(calls, outs, replays=2):
    """Run `calls` once on a side stream (first-call set-up), zero the outputs, capture the
    calls into a graph, replay it, and return the graph's outputs."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        calls()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    for t in outs:
        t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        calls()
    torch.cuda.synchronize()
    assert all(int(torch.count_nonzero(t)) == 0 for t in outs), "capture must not run the work"
    for _ in range(replays):
        g.replay()
    torch.cuda.synchronize()
    return g


def test_single_signal_calls_replay(B):
    p = synth.workload(1)
    ref = oracle.Operator(p.N, p.M, p.op_seed)
    _, y = measurements(p, ref)
    op = B.Operator(p.N, p.M, p.op_seed)
    yd = to_dev(y)
    x = to_dev(np.random.default_rng(0).standard_normal(p.N).astype(np.float32))
    s_direct, k_direct = op.recover(yd, p.K, "omp", 1e-6, 100)
    a_direct = op.apply(x)
    t_direct = op.apply_t(yd)
    torch.cuda.synchronize()
    s_out = torch.empty_like(s_direct)
    k_out = torch.empty(p.K, dtype=torch.int32, device=yd.device)
    a_out = torch.empty_like(a_direct)
    t_out = torch.empty_like(t_direct)

    def calls():
        op.recover(yd, p.K, "omp", 1e-6, 100, s_out, k_out)
        op.apply(x, a_out)
        op.apply_t(yd, t_out)
    capture_and_replay(calls, [s_out, k_out, a_out, t_out])
    assert torch.equal(s_out, s_direct) and torch.equal(k_out, k_direct)
    assert torch.equal(a_out, a_direct) and torch.equal(t_out, t_direct)
    want = oracle.greedy.recover(ref, y.astype(np.float64), p.K, "omp")
    assert rel(s_out.cpu().numpy(), want["s"]) <= SHAT_TOL


@pytest.mark.parametrize("impl", ["cluster", "streamed"])
def test_batched_operator_replays(B, impl):
    N, M, nb = 1 << 16, 1 << 14, 150        # more vectors than one parameter chunk of tasks
    op = B.Operator(N, M, 7)
    op.set_batched_impl(impl)
    g = np.random.default_rng(1)
    X = to_dev(g.standard_normal((nb, N)).astype(np.float32))
    U = to_dev(g.standard_normal((nb, M)).astype(np.float32))
    y_direct = op.apply_batched(X)
    x_direct = op.apply_t_batched(U)
    torch.cuda.synchronize()
    y_out, x_out = torch.empty_like(y_direct), torch.empty_like(x_direct)

    def calls():
        op.apply_batched(X, y_out)
        op.apply_t_batched(U, x_out)
    capture_and_replay(calls, [y_out, x_out])
    assert torch.equal(y_out, y_direct) and torch.equal(x_out, x_direct)
    ref = oracle.Operator(N, M, 7)
    assert rel(y_out[149].cpu().numpy(), ref.apply(X[149].cpu().numpy().astype(np.float64))) <= 1e-5


def test_batched_recovery_over_two_cluster_sizes_and_ls_replay(B):
    g = np.random.default_rng(2)
    cases = [(1 << 12, 1 << 10, 40, "omp"), (1 << 12, 1 << 10, 60, "sp"), (1 << 16, 1 << 14, 300, "sp")]
    ops, refs, ys = [], [], []
    for i, (N, M, K, algo) in enumerate(cases):
        refs.append(oracle.Operator(N, M, 100 + i))
        ops.append(B.Operator(N, M, 100 + i))
        s = synth.sparse_gaussian(N, K, 200 + i)
        ys.append(to_dev(refs[-1].apply(s).astype(np.float32)))
    Ks = [c[2] for c in cases]
    algos = [c[3] for c in cases]
    s_direct, k_direct = B.recover_batched(ops, ys, Ks, algos, 1e-6, 200)
    S = torch.from_numpy(np.sort(g.choice(1 << 16, 500, replace=False)).astype(np.int32)).cuda()
    Sb = S[None, :].repeat(3, 1).contiguous()
    Yb = to_dev(g.standard_normal((3, 1 << 14)).astype(np.float32))
    ls_direct = ops[2].ls_solve(Sb, Yb, 1e-7, 300)
    torch.cuda.synchronize()
    s_outs = [torch.empty_like(t) for t in s_direct]
    k_outs = [torch.empty(max(k, 1), dtype=torch.int32, device=t.device) for k, t in zip(Ks, s_direct)]
    ls_out = torch.empty_like(ls_direct)

    def calls():
        B.recover_batched(ops, ys, Ks, algos, 1e-6, 200, s_outs, k_outs)
        ops[2].ls_solve(Sb, Yb, 1e-7, 300, ls_out)
    capture_and_replay(calls, s_outs + k_outs + [ls_out])
    for a, b in zip(s_outs, s_direct):
        assert torch.equal(a, b)
    for a, b, k in zip(k_outs, k_direct, Ks):
        assert torch.equal(a[:k], b)
    assert torch.equal(ls_out, ls_direct)
    for i, (N, M, K, algo) in enumerate(cases):
        want = oracle.greedy.recover(refs[i], ys[i].cpu().numpy().astype(np.float64), K, algo)
        assert rel(s_outs[i].cpu().numpy(), want["s"]) <= SHAT_TOL


def test_cooperative_grid_recovery_replays(B):
    N, M, K = 1 << 19, 1 << 17, 200
    ref = oracle.Operator(N, M, 31)
    op = B.Operator(N, M, 31)
    s = synth.sparse_gaussian(N, K, 32)
    yd = to_dev(ref.apply(s).astype(np.float32))
    s_direct, k_direct = op.recover(yd, K, "omp", 1e-6, 100)
    torch.cuda.synchronize()
    s_out = torch.empty_like(s_direct)
    k_out = torch.empty(K, dtype=torch.int32, device=yd.device)
    capture_and_replay(lambda: op.recover(yd, K, "omp", 1e-6, 100, s_out, k_out), [s_out, k_out])
    op.sync()
    assert torch.equal(s_out, s_direct) and torch.equal(k_out, k_direct)
    assert rel(s_out.cpu().numpy(), s) <= 1e-4


def test_launch_counter(B):
    """cs_launch_count: one launch per single-signal call, a task-table upload plus one engine
    launch for a batch of several signals of one cluster size, one streamed-operator launch."""
    N, M = 1 << 12, 1 << 10
    op = B.Operator(N, M, 5)
    y = to_dev(np.random.default_rng(3).standard_normal(M).astype(np.float32))
    torch.cuda.synchronize()
    n0 = B.launch_count()
    op.recover(y, 10, "omp", 1e-6, 100)
    assert B.launch_count() - n0 == 1
    n0 = B.launch_count()
    B.recover_batched([op, op, op], [y, y, y], [10, 10, 10], ["omp", "sp", "ompr"], 1e-6, 100)
    assert B.launch_count() - n0 == 2
    big = B.Operator(1 << 16, 1 << 14, 6)
    big.set_batched_impl("streamed")
    X = torch.randn((4, 1 << 16), device="cuda")
    n0 = B.launch_count()
    big.apply_batched(X)
    assert B.launch_count() - n0 == 1
    torch.cuda.synchronize()
