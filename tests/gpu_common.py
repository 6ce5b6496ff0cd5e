"""Helpers shared by the GPU parity tests (inputs from synth, expected values from the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

APPLY_TOL = 1e-5     # rel L2 of one FP32 A / A^T application vs FP64 (derivation in the design notes)
SHAT_TOL = 1e-4      # rel L2 of the recovered s_hat vs the FP64 oracle


def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def measurements(problem, ref_op):
    """y in FP32: formed in FP64 by the oracle (plus seeded noise), rounded once."""
    s = problem.signal()
    y = problem.add_noise(ref_op.apply(s))
    return s, y.astype(np.float32)


def recover_traced(op, y, K, algo, cg_tol=1e-6, cg_maxit=100, ompr_l=1):
    """One recovery through the C ABI with the selection trace on.  y: numpy FP32 or a CUDA
    tensor.  Returns numpy (s_hat, support), the statistics and the trace."""
    from oracle import replay
    tr = torch.zeros(replay.trace_words(op.N, K, algo, ompr_l=ompr_l), dtype=torch.int32, device=dev())
    op.set_trace(tr)
    yd = y if isinstance(y, torch.Tensor) else to_dev(np.asarray(y, dtype=np.float32))
    s, supp = op.recover(yd, K, algo, cg_tol, cg_maxit)
    st = op.stats()
    op.set_trace(None)
    return s.cpu().numpy(), supp.cpu().numpy(), st, tr.cpu().numpy()


def replay_parity(op, ref_op, y, K, algo, cg_tol=1e-6, cg_maxit=100, shat_tol=SHAT_TOL, ompr_l=1, cg_rel=None,
                  **okw):
    """Recover on the GPU with the trace on, replay the FP64 oracle along it and assert
    selection-by-selection parity (exact above the 1e-3 margin and the FP32 resolution that the
    CG tolerance sets; cg_rel overrides the tolerance for absolute-xi runs), the same final
    support and s_hat within shat_tol; the device's near-tie statistics must match its trace.  Returns
    (report, s_hat, support, stats, replayed oracle result)."""
    from oracle import replay
    s, supp, st, tr = recover_traced(op, y, K, algo, cg_tol, cg_maxit, ompr_l)
    assert st["status"] == 0
    kw = dict(okw)
    if algo == "ompr" and ompr_l > 1:
        kw["l"] = ompr_l
    yh = y.cpu().numpy() if isinstance(y, torch.Tensor) else y
    rep, ref = replay.check_recovery(ref_op, np.asarray(yh, dtype=np.float64), K, algo, tr, s, supp, shat_tol,
                                     stats=st, cg_tol=cg_tol if cg_rel is None else cg_rel, **kw)
    return rep, s, supp, st, ref
