"""GPU check of cs_recover_noalloc, the recovery entry point for callers that cannot allocate
device memory (its scratch is the library's fixed device array).  Collected last on purpose.

Two calls in a row go through the C ABI; each must reproduce what cs_recover returns for the
same input within the recovery tolerance used by the other GPU tests (the kernel and its
arithmetic are the same, so the results are expected to be identical)."""
import numpy as np
import pytest

import oracle
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, measurements, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_recover_on_two_calls_in_a_row():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    # call 1: OMP at the N = 4096 workload (one CTA); call 2: SP at N = 2^16 (a 4-CTA cluster,
    # the largest size the fixed scratch holds)
    problems = [synth.workload(1), synth.Problem(1 << 16, 1 << 14, 800, "sp", 0x77001, 0x77002, 0x77003, 1e-3)]
    cases = []
    for p in problems:
        ref_op = oracle.Operator(p.N, p.M, p.op_seed)
        _, y = measurements(p, ref_op)
        op = binding.Operator(p.N, p.M, p.op_seed)
        yd = to_dev(y)
        s_out = torch.empty(p.N, dtype=torch.float32, device=yd.device)
        k_out = torch.empty(p.K, dtype=torch.int32, device=yd.device)
        cases.append((p, op, yd, s_out, k_out))
    got = []
    for p, op, yd, s_out, k_out in cases:                 # two no-alloc calls back to back
        op.recover_noalloc(yd, p.K, p.algo, 1e-6, 200, s_out, k_out)
        got.append((s_out.clone(), k_out.clone()))
    torch.cuda.synchronize()
    for (p, op, yd, _, _), (s_na, k_na) in zip(cases, got):
        s_ref, k_ref = op.recover(yd, p.K, p.algo, 1e-6, 200)
        torch.cuda.synchronize()
        assert np.array_equal(k_na.cpu().numpy(), k_ref.cpu().numpy()), p
        assert rel(s_na.cpu().numpy(), s_ref.cpu().numpy()) <= SHAT_TOL, p


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1509_03979_gb300 import binding
    op = binding.Operator(1 << 17, 1 << 15, 5)
    y = torch.zeros(1 << 15, dtype=torch.float32, device="cuda")
    with pytest.raises(RuntimeError, match="65536"):
        op.recover_noalloc(y, 10, "omp")


def test_noalloc_allocates_nothing_and_matches_the_oracle():
    """After a warm-up call, two more calls leave the device's free memory and the torch
    allocator's counters unchanged (the call allocates nothing), and the result matches the FP64
    oracle selection by selection (its trace replayed) with s_hat within the recovery tolerance."""
    from paper_1509_03979_gb300 import binding
    from oracle import replay
    binding.lib()
    p = synth.Problem(1 << 15, 1 << 13, 400, "sp", 0x78001, 0x78002, 0x78003, 1e-3)
    ref_op = oracle.Operator(p.N, p.M, p.op_seed)
    _, y = measurements(p, ref_op)
    op = binding.Operator(p.N, p.M, p.op_seed)
    yd = to_dev(y)
    s_out = torch.empty(p.N, dtype=torch.float32, device=yd.device)
    k_out = torch.empty(p.K, dtype=torch.int32, device=yd.device)
    tr = torch.zeros(replay.trace_words(p.N, p.K, "sp"), dtype=torch.int32, device=yd.device)
    op.set_trace(tr)
    op.recover_noalloc(yd, p.K, "sp", 1e-6, 200, s_out, k_out)      # warm-up: first call on the device
    torch.cuda.synchronize()
    keys = ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.allocated")
    before = {k: torch.cuda.memory_stats().get(k, 0) for k in keys}
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        op.recover_noalloc(yd, p.K, "sp", 1e-6, 200, s_out, k_out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert {k: torch.cuda.memory_stats().get(k, 0) for k in keys} == before
    op.set_trace(None)
    replay.check_recovery(ref_op, y.astype(np.float64), p.K, "sp", tr.cpu().numpy(), s_out.cpu().numpy(),
                          k_out.cpu().numpy(), SHAT_TOL)
