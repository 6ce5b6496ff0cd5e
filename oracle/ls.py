"""Oracle least-squares solvers on a fixed support (test infrastructure only).

Sec. II step 3 defines the sub-problem s = (A_S^T A_S)^{-1} A_S^T y, the minimiser of
||y - A_S s||_2.  Theorems 1-2 (Sec. III-B, III-C) show that the weighted problem
min ||y - A W_S theta|| (Eq. 9) and its normal-equation form min ||W^T A^T (y - A W theta)||
(Eq. 10) have the same entries on S; Algorithm 1 solves the latter by conjugate gradients on
H = W^T A^T A W with b = W^T A^T y.  On the support, H restricted to S is A_S^T A_S (proof of
Theorem 5), so CG is run on |S|-long vectors.

Solvers:
  * `ls_qr`        -- Householder QR of the dense A_S (the closed form; ground truth).
  * `ls_cholesky`  -- Cholesky of the Gram matrix A_S^T A_S (independent cross-check).
  * `cg_alg1`      -- Algorithm 1's CG with the loop test read as "while ||r_j|| > tol"
                      (the printed "<=" cannot be meant: the loop would never start).
  * `GrowingCholesky` -- the Cholesky route for a support that only grows (OMP): the Gram
                      matrix gains one row and column per step, A_S^T a_t = (A^T A e_t)[S] is
                      one A and one A^T application, and the factor is extended by one row
                      instead of refactored.  Same closed form as `ls_cholesky`.
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


def ls_cg(op, S, y, tol=1e-13, maxit=None, x0=None):
    """LS(S) through CG in FP64 to a relative residual `tol` (O-fast tier for large |S|).
    x0 (optional, |S| entries) is a starting point: the solution is unique, so a start only
    changes the number of steps, not what the solver converges to."""
    S = np.asarray(S, dtype=np.int64)
    b = op.apply_t(y)[S]
    x, _, _ = cg_alg1(op, S, b, tol, maxit if maxit is not None else 10 * len(S) + 50, x0=x0)
    return x


def ls(op, S, y, method="auto", x0=None):
    """LS(S): closed form when A_S fits comfortably, else FP64 CG to 1e-13 (started at x0 when
    given)."""
    S = np.asarray(S, dtype=np.int64)
    if len(S) == 0:
        return np.zeros(0)
    if method == "auto":
        method = "qr" if op.M * len(S) <= 4_000_000 else "cg"
    if method == "qr":
        return ls_qr(op.columns(S), np.asarray(y, dtype=np.float64))
    if method == "cholesky":
        return ls_cholesky(op.columns(S), np.asarray(y, dtype=np.float64))
    return ls_cg(op, S, y, x0=x0)


class GrowingCholesky:
    """LS(S) for a support that gains one index per step (OMP), by the Cholesky factor
    G = L L^T of the Gram matrix G = A_S^T A_S kept in the order the indices arrived.

    Adding index t: g = A_S^T a_t = (A^T (A e_t))[S] (one application each of A and A^T),
    gamma = ||a_t||^2 = (A^T A e_t)[t]; the new row of L is l = L^{-1} g and its diagonal
    entry sqrt(gamma - l.l).  LS(S) is then L^{-T} L^{-1} (A^T y)[S] -- the closed form of
    `ls_cholesky`, built incrementally."""

    def __init__(self, op, y, capacity=16):
        self.op = op
        self.aty = op.apply_t(np.asarray(y, dtype=np.float64))
        self.order = []
        self.L = np.zeros((capacity, capacity))   # the leading k x k block is the factor

    def add(self, t):
        e = np.zeros(self.op.N)
        e[t] = 1.0
        col = self.op.apply_t(self.op.apply(e))
        k = len(self.order)
        if k == self.L.shape[0]:                  # grow the storage, keep the factor
            big = np.zeros((2 * k, 2 * k))
            big[:k, :k] = self.L
            self.L = big
        Lk = self.L[:k, :k]
        g = col[np.asarray(self.order, dtype=np.int64)] if k else np.zeros(0)
        l = sla.solve_triangular(Lk, g, lower=True) if k else np.zeros(0)
        diag2 = col[t] - float(l @ l)
        if not diag2 > 0.0:
            raise np.linalg.LinAlgError("A_S lost full column rank")
        self.L[k, :k] = l
        self.L[k, k] = np.sqrt(diag2)
        self.order.append(int(t))

    def solve(self):
        """(S sorted ascending, LS(S) in that order)."""
        o = np.asarray(self.order, dtype=np.int64)
        k = len(o)
        Lk = self.L[:k, :k]
        z = sla.solve_triangular(Lk, self.aty[o], lower=True)
        x = sla.solve_triangular(Lk, z, lower=True, trans="T")
        perm = np.argsort(o)
        return o[perm], x[perm]
