"""GPU: the paper's own workload (Sec. IV-A: M = N/4, K = N/16, sigma_eta = 0.01) with its CG
stopping rules (Algorithm 1 with an absolute xi, and exact precision = at most |S| steps,
Theorem 5), against the FP64 oracle's exact least squares."""
import numpy as np
import pytest

import oracle
from oracle import greedy
from paper_1509_03979_gb300 import synth
from tests.gpu_common import SHAT_TOL, rel, replay_parity, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def _problem(N, seed):
    M, K, s, noise = synth.paper_workload(N, seed)
    ref = oracle.Operator(N, M, seed)
    y = (ref.apply(s) + noise).astype(np.float32)
    return M, K, s, ref, y


@pytest.mark.parametrize("algo", ["omp", "sp", "ompr"])
@pytest.mark.parametrize("N", [1 << 11, 1 << 12])
@pytest.mark.parametrize("mode", ["xi=1e-5", "exact"])
def test_paper_workload_matches_exact_ls(B, algo, N, mode):
    seed = 0x1509 + N
    M, K, s, ref, y = _problem(N, seed)
    op = B.Operator(N, M, seed)
    op.set_cg_tol_mode("absolute")
    tol, maxit = (1e-5, 0) if mode == "xi=1e-5" else (0.0, 0)
    # selection by selection against the oracle (exact LS); the s_hat bound:
    # an absolute stop at ||r|| <= xi leaves ||x - x*|| <= xi / lambda_min(A_S^T A_S); with
    # lambda_min >= (1 - sqrt(2K/M))^2 = 0.086 here that is < 1.2e-4 absolute, ~1e-5 relative;
    # exact precision stops at the FP32 floor ||r|| <= 1e-6 ||b||, ~1e-5 relative
    rel_tol = max(tol / (np.sqrt(M / N) * np.linalg.norm(y)), 1e-6)   # the absolute xi relative to ||b||
    rep, got, supp, st, want = replay_parity(op, ref, y, K, algo, tol, maxit, cg_rel=rel_tol)
    if algo == "omp" and mode == "exact":
        # Theorem 5: the solve on i columns takes at most i steps
        assert st["cg_iters_total"] <= K * (K + 1) // 2


def test_absolute_xi_stops_earlier_than_exact(B):
    N = 1 << 12
    M, K, s, ref, y = _problem(N, 77)
    op = B.Operator(N, M, 77)
    op.set_cg_tol_mode("absolute")
    op.recover(to_dev(y), K, "sp", 1e-5, 0)
    loose = op.stats()["cg_iters_total"]
    op.recover(to_dev(y), K, "sp", 0.0, 0)
    exact = op.stats()["cg_iters_total"]
    assert loose < exact
    op.set_cg_tol_mode("relative")
    op.recover(to_dev(y), K, "sp", 1e-6, 100)
    assert op.stats()["status"] == 0


def test_cg_tol_mode_rejects_unknown(B):
    op = B.Operator(1024, 256, 1)
    with pytest.raises(KeyError):
        op.set_cg_tol_mode("sloppy")
    from paper_1509_03979_gb300 import binding
    assert binding.lib().cs_op_set_cg_tol_mode(op._h, 7) != 0


@pytest.mark.parametrize("N,M,K,l", [(4096, 1024, 64, 16), (1 << 12, 1 << 10, 1 << 8, 64), (1 << 15, 4000, 300, 300)])
def test_ompr_l_matches_oracle(B, N, M, K, l):
    """OMPR(l): same supports and rounds as the FP64 oracle's OMPR(l), s_hat within 1e-4."""
    seed = 0x0A11 + N + l
    p = synth.Problem(N=N, M=M, K=K, algo="ompr", op_seed=seed, signal_seed=seed + 1, noise_seed=seed + 2,
                      noise_rel=1e-3)
    ref = oracle.Operator(N, M, seed)
    y = p.add_noise(ref.apply(p.signal())).astype(np.float32)
    op = B.Operator(N, M, seed)
    op.set_ompr_replacements(l)
    rep, s_hat, supp, st, want = replay_parity(op, ref, y, K, "ompr", 1e-6, 200, ompr_l=l)
    assert st["outer_iters"] == want["iters"]


def test_ompr_replacements_rejects_zero(B):
    op = B.Operator(1024, 256, 1)
    with pytest.raises(RuntimeError):
        op.set_ompr_replacements(0)
