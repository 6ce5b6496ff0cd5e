"""GPU parity at the benchmark's full size and launch configuration: SP + CG-LS at N = 2^18,
M = 65 536, K = 6 554 with 1e-3 noise, one batched launch over 8 signals per resident cluster
(the configuration bench.py times, same seeds and CG settings), three of them checked against
the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import greedy
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CG_TOL, CG_MAXIT = 5e-6, 100   # the benchmark's settings for this workload


def test_sp_full_size_batched_matches_oracle():
    from paper_1509_03979_gb300 import binding
    p = synth.workload(2)
    op = binding.Operator(p.N, p.M, p.op_seed)
    B = 8 * op.concurrency()
    S = np.stack([synth.sparse_gaussian(p.N, p.K, p.signal_seed + 7919 * i) for i in range(B)]).astype(np.float32)
    noise = np.stack([synth.normals(p.noise_seed + 7919 * i, p.M) for i in range(B)]).astype(np.float32)
    Yc = op.apply_batched(torch.from_numpy(S).cuda())
    sigma = p.noise_rel * torch.linalg.vector_norm(Yc, dim=1, keepdim=True) / np.sqrt(p.M)
    Y = (Yc + sigma * torch.from_numpy(noise).cuda()).contiguous()
    s_b, k_b, st = binding.recover_batched([op] * B, [Y[b] for b in range(B)], [p.K] * B, ["sp"] * B,
                                           CG_TOL, CG_MAXIT, want_stats=True)
    assert all(x["status"] == 0 for x in st)
    ref = oracle.Operator(p.N, p.M, p.op_seed)
    for b in (0, B // 2, B - 1):
        want = greedy.sp(ref, Y[b].cpu().numpy().astype(np.float64), p.K)
        assert rel(s_b[b].cpu().numpy(), want["s"]) <= SHAT_TOL, b
        got = set(k_b[b].cpu().numpy().tolist())
        # supports differ only at the oracle's near-ties: at most that many entries
        assert len(got ^ set(want["S"].tolist())) <= 2 * want["near_ties"], b


def test_mixed_batch_full_size_sampled_against_oracle():
    """The full 256-signal mixed batch in one call, as bench.py --workload batched runs it;
    sampled outputs the oracle can recompute quickly: the four smallest-work signals and the
    largest-N SP signal."""
    from paper_1509_03979_gb300 import binding
    probs = synth.batched_workload(B=256)
    ops, ys = [], []
    for p in probs:
        op = binding.Operator(p.N, p.M, p.op_seed)
        yc = op.apply(torch.from_numpy(p.signal().astype(np.float32)).cuda())
        sig = p.noise_rel * torch.linalg.vector_norm(yc) / np.sqrt(p.M)
        ys.append((yc + sig * torch.from_numpy(p.noise_unit().astype(np.float32)).cuda()).contiguous())
        ops.append(op)
    s_b, k_b, st = binding.recover_batched(ops, ys, [p.K for p in probs], [p.algo for p in probs],
                                           CG_TOL, CG_MAXIT, want_stats=True)
    assert all(x["status"] == 0 for x in st)
    work = [p.N * p.K for p in probs]
    sample = list(np.argsort(work)[:4])
    sp_big = [i for i, p in enumerate(probs) if p.algo == "sp"]
    sample.append(max(sp_big, key=lambda i: (probs[i].N, -probs[i].K)))
    for i in sample:
        p = probs[i]
        ref = oracle.Operator(p.N, p.M, p.op_seed)
        want = greedy.recover(ref, ys[i].cpu().numpy().astype(np.float64), p.K, p.algo)
        assert rel(s_b[i].cpu().numpy(), want["s"]) <= SHAT_TOL, (i, p)
