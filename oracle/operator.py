"""Oracle sensing operator A = P_Omega . C_N . diag(d) (test infrastructure only).

Sec. III-A, Eq. 7: the structurally random matrix Phi = D F R with D a row sampler, F an
orthonormal fast transform (the DCT) and R a randomiser.  Here R is the Rademacher sign flip
diag(d), F = C_N the orthonormal DCT-II, D = P_Omega keeps the rows in Omega.  The sparsifying
basis is the identity, so A = Phi and y = A s (Eq. 1-2).  No sqrt(N/M) rescaling is applied,
hence A A^T = I_M.

Sec. III-D lists the operator realisations this follows: "W x" zeroes entries outside the
support, "D x" picks M entries, "F x" is the DCT computed by FFT, "R x" is the randomiser.

Optional sparsifying basis Psi (Sec. III-A, y = Phi Psi s; the image experiment of Sec. IV
uses a DCT basis): with `psi` set, the unknown s holds the coefficients of x = Psi s and the
operator is A = P_Omega C_N R Psi.  psi = "dct": Psi = C_N^T (s are the orthonormal DCT-II
coefficients of x); psi = ("dct2d", n1, n2), n1 n2 = N: x is the row-major flattening of
C_{n1}^T S C_{n2} for the n1 x n2 coefficient array S, the separable basis Psi_2 (x) Psi_1.
Psi is orthonormal in both cases, so A A^T = I_M still holds.
"""
import numpy as np

from . import dct as _dct
from . import rng as _rng


class Operator:
    """A in R^{M x N}; `fast=True` applies C_N via FFT (O-fast), else by the O(N^2) sum."""

    def __init__(self, N, M, seed, fast=True, randomizer="signs", psi=None):
        """randomizer 'signs': R = diag(d) (A = P_Omega C_N diag(d)); 'perm': R the paper's random
        permutation, (R x)_n = x[perm[n]], no signs (A = P_Omega C_N Pi); 'none': R = I (for
        closed-form checks only).  psi: None, "dct" or ("dct2d", n1, n2), see the module text."""
        if N < 2:
            raise ValueError("N must be >= 2")   # any N: the FFT step and the draws take any length
        self.N, self.M, self.seed = int(N), int(M), int(seed)
        self.omega = _rng.omega(N, M, seed)
        self.fast = fast
        if psi is not None and psi != "dct":
            kind, n1, n2 = psi
            if kind != "dct2d" or n1 * n2 != N:
                raise ValueError("psi must be None, 'dct' or ('dct2d', n1, n2) with n1 n2 = N")
        self.psi = psi
        if randomizer == "none":
            self.d = np.ones(N)
            self.perm = None
            self.iperm = None
        elif randomizer == "perm":
            self.d = np.ones(N)
            self.perm = _rng.perm(N, seed)
            self.iperm = np.empty(N, dtype=np.int64)
            self.iperm[self.perm] = np.arange(N)
        else:
            self.d = _rng.signs(N, seed)
            self.perm = None
            self.iperm = None

    # --- transforms -------------------------------------------------------------------
    def _c(self, x):
        return _dct.dct2_fast(x) if self.fast else _dct.dct2_naive(x)

    def _ct(self, X):
        return _dct.dct3_fast(X) if self.fast else _dct.dct3_naive(X)

    # --- the sparsifying basis --------------------------------------------------------
    def _psi(self, s):
        """x = Psi s (identity when psi is None)."""
        s = np.asarray(s, dtype=np.float64)
        if self.psi is None:
            return s
        if self.psi == "dct":
            return self._ct(s)
        _, n1, n2 = self.psi
        S = s.reshape(s.shape[:-1] + (n1, n2))
        S = _dct.dct3_naive(S) if not self.fast else _dct.dct3_fast(S)              # along n2
        S = np.swapaxes(_dct.dct3_fast(np.swapaxes(S, -1, -2)) if self.fast
                        else _dct.dct3_naive(np.swapaxes(S, -1, -2)), -1, -2)        # along n1
        return S.reshape(s.shape)

    def _psi_t(self, x):
        """Psi^T x."""
        x = np.asarray(x, dtype=np.float64)
        if self.psi is None:
            return x
        if self.psi == "dct":
            return self._c(x)
        _, n1, n2 = self.psi
        X = x.reshape(x.shape[:-1] + (n1, n2))
        X = _dct.dct2_naive(X) if not self.fast else _dct.dct2_fast(X)
        X = np.swapaxes(_dct.dct2_fast(np.swapaxes(X, -1, -2)) if self.fast
                        else _dct.dct2_naive(np.swapaxes(X, -1, -2)), -1, -2)
        return X.reshape(x.shape)

    # --- A and A^T (Sec. III-D operator list) --------------------------------------------
    def apply(self, x):
        """A x = (C_N (d * Psi x))[Omega], or (C_N (Psi x)[perm])[Omega] for the permutation
        randomiser (Psi = I unless psi is set)."""
        x = self._psi(x)
        if self.perm is not None:
            return self._c(x[..., self.perm])[..., self.omega]
        return self._c(self.d * x)[..., self.omega]

    def apply_t(self, u):
        """A^T u = d * C_N^T (P_Omega^T u)."""
        u = np.asarray(u, dtype=np.float64)
        full = np.zeros(u.shape[:-1] + (self.N,))
        full[..., self.omega] = u
        w = self._ct(full)
        if self.perm is not None:
            out = np.empty_like(w)
            out[..., self.perm] = w
            return self._psi_t(out)
        return self._psi_t(self.d * w)

    def columns(self, S):
        """Dense A_S (M x |S|) from the closed form A[m, j] = d_j w_{Omega_m} cos(pi (2j+1) Omega_m / (2N))
        (with a basis Psi: A applied to the basis vectors Psi e_j)."""
        S = np.asarray(S, dtype=np.int64)
        if self.psi is not None:
            E = np.zeros((len(S), self.N))
            E[np.arange(len(S)), S] = 1.0
            return self.apply(E).T
        k = self.omega[:, None].astype(np.float64)
        pos = S if self.perm is None else self.iperm[S]   # DCT input index of each column
        j = pos[None, :].astype(np.float64)
        w = _dct.weights(self.N)[self.omega][:, None]
        return self.d[S][None, :] * w * np.cos(np.pi * (2.0 * j + 1.0) * k / (2.0 * self.N))

    def dense(self):
        return self.columns(np.arange(self.N))

    def apply_support(self, S, v):
        """A W_S theta for theta supported on S with values v (Eq. 8's weighting)."""
        x = np.zeros(self.N)
        x[np.asarray(S, dtype=np.int64)] = v
        return self.apply(x)
