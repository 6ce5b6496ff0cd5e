"""Oracle least-squares solvers on a fixed support (test infrastructure only).

Sec. II step 3 defines the sub-problem s = (A_S^T A_S)^{-1} A_S^T y, the minimiser of
||y - A_S s||_2.  Theorems 1-2 (Sec. III-B, III-C) show that the weighted problem
min ||y - A W_S theta|| (Eq. 9) and its normal-equation form min ||W^T A^T (y - A W theta)||
(Eq. 10) have the same entries on S; Algorithm 1 solves the latter by conjugate gradients on
H = W^T A^T A W with b = W^T A^T y.  On the support, H restricted to S is A_S^T A_S (proof of
Theorem 5), so CG is run on |S|-long vectors.

Three solvers:
  * `ls_qr`        -- Householder QR of the dense A_S (the closed form; ground truth).
  * `ls_cholesky`  -- Cholesky of the Gram matrix A_S^T A_S (independent cross-check).
  * `cg_alg1`      -- Algorithm 1's CG with the loop test read as "while ||r_j|| > tol"
                      (the printed "<=" cannot be meant: the loop would never start).
"""
import numpy as np
import scipy.linalg as sla


def ls_qr(AS, y):
    """argmin ||y - AS s||_2 by Householder QR (numpy/LAPACK geqrf)."""
    Q, R = np.linalg.qr(AS, mode="reduced")
    return sla.solve_triangular(R, Q.T @ y, lower=False)


def ls_cholesky(AS, y):
    G = AS.T @ AS
    c = sla.cho_factor(G, lower=True)
    return sla.cho_solve(c, AS.T @ y)


def gram_apply(op, S, p):
    """H p on the support: (A^T A (scatter p on S))[S]  -- the matvec of Algorithm 1."""
    return op.apply_t(op.apply_support(S, p))[np.asarray(S, dtype=np.int64)]


def cg_alg1(op, S, b, tol, maxit, x0=None, absolute=False):
    """Algorithm 1 CG on A_S^T A_S x = b (compressed to |S| entries).

    Stops when ||r_j|| <= tol * ||b|| (relative, default) or ||r_j|| <= tol (absolute=True), or
    after `maxit` steps.  Returns (x, iterations, final ||r||).
    """
    S = np.asarray(S, dtype=np.int64)
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros(len(S)) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - gram_apply(op, S, x) if x0 is not None else b.copy()
    d = r.copy()
    rr = float(r @ r)
    stop = tol if absolute else tol * float(np.sqrt(b @ b))
    j = 0
    while np.sqrt(rr) > stop and j < maxit:
        Hd = gram_apply(op, S, d)
        alpha = rr / float(d @ Hd)
        x = x + alpha * d
        r = r - alpha * Hd
        rr_new = float(r @ r)
        beta = rr_new / rr
        d = r + beta * d
        rr = rr_new
        j += 1
    return x, j, float(np.sqrt(rr))


def ls_cg(op, S, y, tol=1e-13, maxit=None):
    """LS(S) through CG in FP64 to a relative residual `tol` (O-fast tier for large |S|)."""
    S = np.asarray(S, dtype=np.int64)
    b = op.apply_t(y)[S]
    x, _, _ = cg_alg1(op, S, b, tol, maxit if maxit is not None else 10 * len(S) + 50)
    return x


def ls(op, S, y, method="auto"):
    """LS(S): closed form when A_S fits comfortably, else FP64 CG to 1e-13."""
    S = np.asarray(S, dtype=np.int64)
    if len(S) == 0:
        return np.zeros(0)
    if method == "auto":
        method = "qr" if op.M * len(S) <= 4_000_000 else "cg"
    if method == "qr":
        return ls_qr(op.columns(S), np.asarray(y, dtype=np.float64))
    if method == "cholesky":
        return ls_cholesky(op.columns(S), np.asarray(y, dtype=np.float64))
    return ls_cg(op, S, y)
