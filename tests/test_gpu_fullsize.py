"""GPU parity at full size, in the launch configurations bench.py times, selection by selection
against the FP64 oracle (the oracle replays each GPU trajectory and continues with the GPU's
choice only at near-ties):

  * SP + CG-LS at N = 2^18, M = 65 536, K = 6 554 with 1e-3 noise: one batched launch over 8
    signals per resident cluster (the bench's seeds and CG settings); 8 signals spread over the
    batch are replayed in full;
  * the 256-signal mixed batch (N = 2^12 .. 2^18, OMP / SP) in one call: every SP signal and
    every OMP signal with K <= 4096 and N <= 2^16 replayed in full; the remaining OMP signals
    (N >= 2^17, or K > 4096, whose full FP64 replay would take CPU-hours) checked at three
    selections each (the first, the middle and the last) from the GPU's own state, plus the
    final s_hat against the FP64 least-squares solution on the GPU's support.

The replays run in a spawn-started process pool (one numpy thread per worker)."""
import numpy as np
import pytest

from paper_1509_03979_gb300 import synth
from oracle import replay
from tests.gpu_common import SHAT_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CG_TOL, CG_MAXIT = 2e-5, 100   # the benchmark's settings for these batched workloads


def _trace(op, K, algo):
    tr = torch.zeros(replay.trace_words(op.N, K, algo), dtype=torch.int32, device="cuda")
    op.set_trace(tr)
    return tr


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
    sample = sorted(set(np.linspace(0, B - 1, 8).round().astype(int).tolist()))
    ops, traces = [op] * B, {}
    for b in sample:                       # same operator, own handle for its own trace
        ops[b] = binding.Operator(p.N, p.M, p.op_seed)
        traces[b] = _trace(ops[b], p.K, "sp")
    s_b, k_b, st = binding.recover_batched(ops, [Y[b] for b in range(B)], [p.K] * B, ["sp"] * B,
                                           CG_TOL, CG_MAXIT, want_stats=True)
    torch.cuda.synchronize()
    assert all(x["status"] == 0 for x in st)
    jobs = [dict(N=p.N, M=p.M, op_seed=p.op_seed, y=Y[b].cpu().numpy().astype(np.float64), K=p.K, algo="sp",
                 trace=traces[b].cpu().numpy(), s=s_b[b].cpu().numpy(), supp=k_b[b].cpu().numpy(),
                 stats=st[b], shat_tol=SHAT_TOL, cg_tol=CG_TOL, index=b) for b in sample]
    reps = replay.run_pool(replay.replay_job, jobs)
    assert len(reps) == len(sample) >= 4
    for r in reps:
        assert r["rel_err"] <= SHAT_TOL and r["selections"] >= 3, r


def _mixed_batch():
    from paper_1509_03979_gb300 import binding
    probs = synth.batched_workload(B=256)
    ops, ys, trs = [], [], []
    for p in probs:
        op = binding.Operator(p.N, p.M, p.op_seed)
        yc = op.apply(torch.from_numpy(p.signal().astype(np.float32)).cuda())
        sig = p.noise_rel * torch.linalg.vector_norm(yc) / np.sqrt(p.M)
        ys.append((yc + sig * torch.from_numpy(p.noise_unit().astype(np.float32)).cuda()).contiguous())
        trs.append(_trace(op, p.K, p.algo))
        ops.append(op)
    return binding, probs, ops, ys, trs


def test_mixed_batch_full_size_against_oracle():
    """The full 256-signal mixed batch in one call, as bench.py times it (config of the
    batched-recovery workload); the coverage is stated in the module docstring."""
    binding, probs, ops, ys, trs = _mixed_batch()
    s_b, k_b, st = binding.recover_batched(ops, ys, [p.K for p in probs], [p.algo for p in probs],
                                           CG_TOL, CG_MAXIT, want_stats=True)
    torch.cuda.synchronize()
    assert all(x["status"] == 0 for x in st)
    full, states, finals = [], [], []
    for i, p in enumerate(probs):
        job = dict(N=p.N, M=p.M, op_seed=p.op_seed, y=ys[i].cpu().numpy().astype(np.float64), K=p.K,
                   algo=p.algo, trace=trs[i].cpu().numpy(), s=s_b[i].cpu().numpy(), supp=k_b[i].cpu().numpy(),
                   stats=st[i], shat_tol=SHAT_TOL, cg_tol=CG_TOL, index=i)
        if p.algo == "sp" or (p.K <= 4096 and p.N <= 1 << 16):
            full.append(job)
        else:
            for t in sorted({0, p.K // 2, p.K - 1}):
                states.append(dict(job, t=t))
            finals.append(job)
    # the longest replays first, so that the pool's tail is short
    full.sort(key=lambda j: -(j["K"] * j["N"]))
    reps = replay.run_pool(replay.replay_job, full)
    assert len(reps) == len(full) and all(r["rel_err"] <= SHAT_TOL for r in reps)
    sreps = replay.run_pool(replay.state_job, states)
    assert len(sreps) == len(states)
    freps = replay.run_pool(replay.final_ls_job, finals)      # s_hat = LS on the returned support
    assert len(freps) == len(finals)
    n_sp = sum(1 for p in probs if p.algo == "sp")
    assert sum(1 for j in full if j["algo"] == "sp") == n_sp
