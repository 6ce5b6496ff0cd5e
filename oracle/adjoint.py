"""Oracle adjoint of the fixed-support least-squares step (test infrastructure only).

On a fixed support S the LS solution is s_S(y) = (A_S^T A_S)^{-1} A_S^T y (Sec. II step 3), a
linear map of y.  Its adjoint maps a cotangent g = dL/ds_S to

    dL/dy = A_S (A_S^T A_S)^{-1} g,

i.e. one solve with the Gram matrix of the normal equations (Eq. 10 restricted to S, as in the
proof of Theorem 5) followed by one forward application of A_S.  The oracle evaluates it in
closed form from the QR factorisation A_S = Q R:  A_S R^{-1} R^{-T} g = Q R^{-T} g.
"""
import numpy as np
import scipy.linalg as sla

from . import ls as _ls


def ls_backward(op, S, g):
    """dL/dy for cotangent g on support S, by dense FP64 QR."""
    AS = op.columns(np.asarray(S, dtype=np.int64))
    Q, R = np.linalg.qr(AS, mode="reduced")
    return Q @ sla.solve_triangular(R, np.asarray(g, dtype=np.float64), trans="T", lower=False)


def ls_backward_cg(op, S, g, tol=1e-13, maxit=None):
    """Same quantity by FP64 CG on the Gram system, then A_S z (the matrix-free route)."""
    S = np.asarray(S, dtype=np.int64)
    z, _, _ = _ls.cg_alg1(op, S, g, tol, maxit if maxit is not None else 10 * len(S) + 50)
    return op.apply_support(S, z)


def loss_grad_y(op, S, y, s_true_S):
    """L(y) = ||s_S(y) - s_true_S||^2 and its exact gradient with respect to y."""
    AS = op.columns(np.asarray(S, dtype=np.int64))
    sS = _ls.ls_qr(AS, np.asarray(y, dtype=np.float64))
    diff = sS - s_true_S
    return float(diff @ diff), ls_backward(op, S, 2.0 * diff)
