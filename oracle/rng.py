"""Oracle's own implementation of the operator's random draws (test infrastructure only).

The structured sensing matrix of Sec. III-A (Eq. 7) needs two random objects: the row sampler
(the paper's D, here the sorted row subset Omega of size M) and the randomiser (here a
Rademacher sign vector d, which replaces the paper's random permutation R).  Both are defined
from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), written here from that published definition:

    gamma = 0x9E3779B97F4A7C15
    mix(z):  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB;
             z ^= z >> 31
    h(x)   = mix(x + gamma)                      (all arithmetic modulo 2**64)
    stream seeded with s: the i-th output (i = 1, 2, ...) is mix(s + i * gamma)

    signs:  d_n = -1 if the top bit of h((seed ^ 0xD1B54A32D192ED03) + n) is set, else +1
    Omega:  partial Fisher-Yates over perm = [0, N): for i = 0..M-1,
            j = i + (u_{i+1} mod (N - i)) with u the stream seeded with seed ^ gamma,
            swap perm[i], perm[j]; Omega = sorted(perm[:M]).

The CUDA library implements the same definition independently; the two share no code.
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
SIGN_SALT = 0xD1B54A32D192ED03
_M64 = (1 << 64) - 1


def mix64(z):
    """SplitMix64 finaliser on Python ints (exact modulo 2**64)."""
    z &= _M64
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) & _M64
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) & _M64
    z ^= z >> 31
    return z


def mix64_np(z):
    """SplitMix64 finaliser on a numpy uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream(seed, count, start=1):
    """Outputs start..start+count-1 of the SplitMix64 stream seeded with `seed`."""
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(seed & _M64) + i * np.uint64(GAMMA)
    return mix64_np(x)


def signs(N, seed):
    """Rademacher randomiser d in {+1,-1}^N (replaces R of Eq. 7)."""
    n = np.arange(N, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64((seed ^ SIGN_SALT) & _M64) + n + np.uint64(GAMMA)
    top = mix64_np(x) >> np.uint64(63)
    return np.where(top == 1, -1.0, 1.0)


def omega(N, M, seed):
    """Sorted row subset Omega (the sampling operator of Eq. 7), |Omega| = M."""
    if not (1 <= M <= N):
        raise ValueError("need 1 <= M <= N")
    u = stream((seed ^ GAMMA) & _M64, M)
    perm = np.arange(N, dtype=np.int64)
    span = (N - np.arange(M, dtype=np.uint64)).astype(np.uint64)
    jump = (u % span).astype(np.int64)
    for i in range(M):
        j = i + int(jump[i])
        perm[i], perm[j] = perm[j], perm[i]
    return np.sort(perm[:M])


PERM_SALT = 0xA0761D6478BD642F


def perm(N, seed):
    """The permutation randomiser R of the SRM (Sec. III-A: a uniform random permutation): a full
    Fisher-Yates shuffle of [0, N) with j = i + (u_{i+1} mod (N - i)), u the SplitMix64 stream
    seeded with seed ^ PERM_SALT; (R x)_n = x[perm[n]]."""
    u = stream((seed ^ PERM_SALT) & _M64, max(N - 1, 0))
    p = np.arange(N, dtype=np.int64)
    span = (N - np.arange(max(N - 1, 0), dtype=np.uint64)).astype(np.uint64)
    jump = (u % span).astype(np.int64)
    for i in range(N - 1):
        j = i + int(jump[i])
        p[i], p[j] = p[j], p[i]
    return p
