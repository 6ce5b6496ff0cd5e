"""Seeded synthetic inputs for tests and benchmarks (no decoder arithmetic lives here).

The paper's experiments use synthetic signals only (Sec. IV-A, Eq. 12: Bernoulli-Gaussian
entries s ~ p N(0, sigma_on^2)).  The workloads below follow that model with the sizes of the
five benchmark workloads; everything is drawn from SplitMix64 streams (Steele, Lea & Flood,
OOPSLA 2014) so that both the CUDA path and the oracle receive bit-identical inputs:

    stream seeded with s: u_i = mix(s + i * 0x9E3779B97F4A7C15), i = 1, 2, ...
    uniform in [0, 1):    (u_i >> 11) * 2**-53
    normals:              Box-Muller on consecutive uniform pairs (1 - U_{2i}, U_{2i+1})
    random positions:     the first K entries of the stable argsort of the u stream

The measurement y = A s itself is NOT formed here: callers compute it with the operator they
are testing (the oracle in tests, the library in the benchmark), so this module holds no part
of the method.
"""
import dataclasses

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1
VALUE_SALT = 0x1000000


def _mix(z):
    with np.errstate(over="ignore"):
        z = z.copy()
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def stream(seed, count):
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed & _M64) + i * np.uint64(GAMMA))


def uniforms(seed, count):
    return (stream(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normals(seed, count):
    n2 = (count + 1) // 2
    u = uniforms(seed, 2 * n2)
    r = np.sqrt(-2.0 * np.log(1.0 - u[0::2]))
    th = 2.0 * np.pi * u[1::2]
    out = np.empty(2 * n2)
    out[0::2] = r * np.cos(th)
    out[1::2] = r * np.sin(th)
    return out[:count]


def positions(seed, N, K):
    """K distinct uniformly random positions in [0, N) (first K of a random permutation)."""
    return np.argsort(stream(seed, N), kind="stable")[:K].astype(np.int64)


def sparse_gaussian(N, K, seed):
    """K-sparse s with N(0,1) values at uniformly random positions (Eq. 12 with sigma_on = 1)."""
    s = np.zeros(N)
    s[positions(seed, N, K)] = normals(seed ^ VALUE_SALT, K)
    return s


def power_law(N, K, seed, tail=1e-4, exponent=1.5):
    """Approximately sparse s: |s| at rank i is i^-1.5 for i <= K and tail * i^-1.5 beyond,
    random signs, ranks placed at a random permutation of the positions."""
    rank = np.arange(1, N + 1, dtype=np.float64)
    mag = rank ** -exponent
    mag[K:] *= tail
    sign = np.where(uniforms(seed ^ VALUE_SALT, N) < 0.5, -1.0, 1.0)
    s = np.empty(N)
    s[positions(seed, N, N)] = sign * mag
    return s


@dataclasses.dataclass
class Problem:
    N: int
    M: int
    K: int
    algo: str            # "omp" | "sp" | "ompr"
    op_seed: int
    signal_seed: int
    noise_seed: int
    noise_rel: float     # sigma = noise_rel * ||y_clean|| / sqrt(M)
    model: str = "gaussian"

    def signal(self):
        if self.model == "powerlaw":
            return power_law(self.N, self.K, self.signal_seed)
        return sparse_gaussian(self.N, self.K, self.signal_seed)

    def noise_unit(self):
        return normals(self.noise_seed, self.M)

    def add_noise(self, y_clean):
        """y = y_clean + sigma * n with sigma = noise_rel * ||y_clean|| / sqrt(M)."""
        y_clean = np.asarray(y_clean, dtype=np.float64)
        if self.noise_rel == 0.0:
            return y_clean.copy()
        sigma = self.noise_rel * np.linalg.norm(y_clean) / np.sqrt(self.M)
        return y_clean + sigma * self.noise_unit()


def workload(c):
    """The five workloads by number: 1 OMP N=4096; 2 SP N=2^18; 3 OMPR N=2^22; 5 LS+adjoint."""
    seeds = dict(op_seed=0x0C5000 + c, signal_seed=0x51600 + c, noise_seed=0x40150 + c)
    if c == 1:
        return Problem(4096, 1024, 64, "omp", noise_rel=0.0, **seeds)
    if c == 2:
        N = 1 << 18
        return Problem(N, N // 4, 6554, "sp", noise_rel=1e-3, **seeds)
    if c == 3:
        N = 1 << 22
        return Problem(N, N // 4, 83886, "ompr", noise_rel=0.0, model="powerlaw", **seeds)
    if c == 5:
        return Problem(1 << 16, 1 << 14, 1024, "sp", noise_rel=0.0, **seeds)
    raise ValueError(c)


def batched_workload(B=256, seed=0x0B000, e_min=12, e_max=18):
    """Mixed batch: N = 2^e, e uniform on {e_min..e_max}; M/N ~ U[0.15, 0.4];
    K/M ~ U[0.05, 0.2]; OMP or SP by a fair coin; N(0,1) nonzeros; sigma = 1e-3 ||y||/sqrt(M)."""
    u = uniforms(seed, 4 * B).reshape(B, 4)
    out = []
    for j in range(B):
        e = e_min + min(int(u[j, 0] * (e_max - e_min + 1)), e_max - e_min)
        N = 1 << e
        M = int(round((0.15 + 0.25 * u[j, 1]) * N))
        K = max(1, int(round((0.05 + 0.15 * u[j, 2]) * M)))
        algo = "sp" if u[j, 3] < 0.5 else "omp"
        base = seed + 3 * (j + 1)
        out.append(Problem(N, M, K, algo, op_seed=base, signal_seed=base + 1,
                           noise_seed=base + 2, noise_rel=1e-3))
    return out


PAPER_SIGMA_ETA = 0.01   # Sec. IV-A: sigma_on = 1, sigma_eta = 0.01 (absolute)


def paper_workload(N, seed):
    """The paper's own simulation setting (Sec. IV-A): M = N/4, K = M/4 = N/16 (p = 0.0625),
    N(0,1) nonzeros at K random positions, and the absolute noise vector sigma_eta * N(0,1) of
    length M that is added to A s.  Returns (M, K, s, noise)."""
    M, K = N // 4, N // 16
    s = sparse_gaussian(N, K, seed)
    noise = PAPER_SIGMA_ETA * normals(seed ^ 0x40150, M)
    return M, K, s, noise
