"""Oracle DCTs (test infrastructure only).

The transform F of Eq. 7 is the orthonormal DCT (Sec. III-A), applied "via FFT" for speed
(Sec. III-D, operator list).  Definition used throughout (orthonormal DCT-II):

    X_k = w_k * sum_n x_n cos(pi (2n+1) k / (2N)),   w_0 = sqrt(1/N),  w_k = sqrt(2/N) (k >= 1)

Its transpose (and inverse, since the matrix is orthonormal) is the orthonormal DCT-III.

Two tiers:
  * `dct_matrix` / `dct2_naive` / `dct3_naive`: the definition written out as an O(N^2) sum.
  * `dct2_fast` / `dct3_fast`: Makhoul's reordering (J. Makhoul, "A fast cosine transform in one
    and two dimensions", IEEE TASSP 1980) with numpy's FFT as the library step:
      v = [x_0, x_2, ..., x_{N-2}, x_{N-1}, ..., x_3, x_1],  V = FFT_N(v),
      X_k = w_k Re(exp(-i pi k / (2N)) V_k).
"""
import numpy as np


def weights(N):
    w = np.full(N, np.sqrt(2.0 / N))
    w[0] = np.sqrt(1.0 / N)
    return w


def dct_matrix(N):
    """Dense orthonormal DCT-II matrix C[k, n] (O-exact tier)."""
    k = np.arange(N)[:, None]
    n = np.arange(N)[None, :]
    return weights(N)[:, None] * np.cos(np.pi * (2 * n + 1) * k / (2.0 * N))


def dct2_naive(x):
    x = np.asarray(x, dtype=np.float64)
    return dct_matrix(x.shape[-1]) @ x


def dct3_naive(X):
    X = np.asarray(X, dtype=np.float64)
    return dct_matrix(X.shape[-1]).T @ X


def dct2_fast(x):
    """Orthonormal DCT-II along the last axis via Makhoul's N-point FFT."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[-1]
    v = np.concatenate([x[..., 0::2], x[..., 1::2][..., ::-1]], axis=-1)
    V = np.fft.fft(v, axis=-1)
    k = np.arange(N)
    return weights(N) * np.real(np.exp(-1j * np.pi * k / (2.0 * N)) * V)


def dct3_fast(X):
    """Orthonormal DCT-III (the transpose of `dct2_fast`) along the last axis.

    Inverts the steps of `dct2_fast`: rebuild the Hermitian spectrum V from X
    (V_k = exp(i pi k/(2N)) (X_k - i X_{N-k}) / w-scaling), inverse FFT, undo the reordering.
    """
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[-1]
    w = weights(N)
    Y = X / w
    Yr = np.zeros_like(Y)
    Yr[..., 1:] = Y[..., :0:-1]          # Yr[k] = Y[N-k] for k >= 1, 0 for k = 0
    k = np.arange(N)
    V = np.exp(1j * np.pi * k / (2.0 * N)) * (Y - 1j * Yr)
    v = np.real(np.fft.ifft(V, axis=-1))
    x = np.empty_like(v)
    h = (N + 1) // 2
    x[..., 0::2] = v[..., :h]
    x[..., 1::2] = v[..., h:][..., ::-1]
    return x
