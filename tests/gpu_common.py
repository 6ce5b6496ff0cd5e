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
