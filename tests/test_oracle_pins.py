"""Pins for the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle function to a library routine, a closed form, an invariant the paper
proves (Theorems 1, 2, 5), brute force, or the ground-truth signal.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.fft as sfft

import oracle
from oracle import adjoint, dct, greedy, ls, rng
from paper_1509_03979_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- generator (Eq. 7 draws)
def test_splitmix64_published_vector():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.startswith("0x")]
    got = [int(v) for v in rng.stream(0, 2)]
    assert got == vals
    # the scalar finaliser agrees with the vectorised one
    assert rng.mix64(0 + rng.GAMMA) == vals[0]


@pytest.mark.parametrize("N,M", [(16, 8), (64, 64), (4096, 1024), (1 << 14, 3000)])
def test_omega_is_sorted_subset(N, M):
    om = rng.omega(N, M, 7)
    assert om.shape == (M,) and om.dtype == np.int64
    assert np.all(np.diff(om) > 0) and om[0] >= 0 and om[-1] < N
    if M == N:
        assert np.array_equal(om, np.arange(N))


def test_omega_uniform_inclusion():
    # each index is included with probability M/N: chi-square over many seeds
    N, M, T = 32, 8, 4000
    counts = np.zeros(N)
    for s in range(T):
        counts[rng.omega(N, M, s)] += 1
    expected = T * M / N
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 70  # 31 dof, p ~ 1e-4


def test_signs_are_rademacher():
    d = rng.signs(1 << 16, 3)
    assert set(np.unique(d)) == {-1.0, 1.0}
    assert abs(d.mean()) < 0.02
    assert not np.array_equal(d, rng.signs(1 << 16, 4))


# ---------------------------------------------------------------- DCT (Sec. III-A, F = DCT)
@pytest.mark.parametrize("N", [2, 4, 16, 64, 1024])
def test_dct_naive_matches_scipy(N):
    x = np.random.default_rng(N).standard_normal(N)
    assert np.allclose(dct.dct2_naive(x), sfft.dct(x, type=2, norm="ortho"), atol=1e-12)
    assert np.allclose(dct.dct3_naive(x), sfft.dct(x, type=3, norm="ortho"), atol=1e-12)


@pytest.mark.parametrize("N", [2, 4, 8, 64, 4096, 1 << 16])
def test_dct_fast_matches_scipy(N):
    x = np.random.default_rng(N + 1).standard_normal(N)
    assert np.allclose(dct.dct2_fast(x), sfft.dct(x, type=2, norm="ortho"), atol=1e-10)
    assert np.allclose(dct.dct3_fast(x), sfft.dct(x, type=3, norm="ortho"), atol=1e-10)


def test_dct_matrix_orthonormal_and_special_vectors():
    N = 128
    C = dct.dct_matrix(N)
    assert np.abs(C @ C.T - np.eye(N)).max() < 1e-12
    e0 = np.zeros(N)
    e0[0] = 1
    assert np.allclose(dct.dct3_fast(e0), np.full(N, 1 / np.sqrt(N)))
    assert np.allclose(dct.dct2_fast(np.full(N, 1 / np.sqrt(N))), e0)
    x = np.random.default_rng(5).standard_normal(N)
    assert np.allclose(dct.dct3_fast(dct.dct2_fast(x)), x, atol=1e-12)


# ---------------------------------------------------------------- operator A = P C D
@pytest.mark.parametrize("N,M", [(16, 8), (256, 64), (1024, 1024)])
def test_operator_rows_orthonormal(N, M):
    op = oracle.Operator(N, M, 11, fast=False)
    A = op.dense()
    assert np.abs(A @ A.T - np.eye(M)).max() < 1e-12          # A A^T = I_M


@pytest.mark.parametrize("fast", [False, True])
def test_operator_apply_matches_dense(fast):
    N, M = 512, 128
    op = oracle.Operator(N, M, 12, fast=fast)
    A = np.stack([dct.dct2_naive(op.d * e)[op.omega] for e in np.eye(N)], axis=1)
    g = np.random.default_rng(0)
    x, u = g.standard_normal(N), g.standard_normal(M)
    assert np.allclose(op.apply(x), A @ x, atol=1e-11)
    assert np.allclose(op.apply_t(u), A.T @ u, atol=1e-11)
    assert np.allclose(op.dense(), A, atol=1e-12)             # closed-form columns


# ---------------------------------------------------------------- least squares (Thm 1, 2, 5)
def _problem(N=1024, M=256, k=40, seed=3):
    op = oracle.Operator(N, M, seed)
    g = np.random.default_rng(seed)
    S = np.sort(g.choice(N, k, replace=False))
    y = g.standard_normal(M)
    return op, S, y


def test_ls_qr_cholesky_lstsq_agree():
    op, S, y = _problem()
    AS = op.columns(S)
    ref = np.linalg.lstsq(AS, y, rcond=None)[0]                # library LS
    assert np.allclose(ls.ls_qr(AS, y), ref, atol=1e-10)
    assert np.allclose(ls.ls_cholesky(AS, y), ref, atol=1e-10)


def test_theorem1_weighted_ls_same_support_entries():
    op, S, y = _problem(N=128, M=64, k=10)
    W = np.zeros(op.N)
    W[S] = 1
    AW = op.dense() * W[None, :]
    theta = np.linalg.pinv(AW) @ y                             # a minimiser of Eq. 9
    assert np.allclose(theta[S], ls.ls_qr(op.columns(S), y), atol=1e-10)


def test_theorem2_cg_matches_closed_form_and_theorem5_bound():
    op, S, y = _problem()
    b = op.apply_t(y)[S]
    x, iters, res = ls.cg_alg1(op, S, b, tol=1e-12, maxit=500)
    assert np.allclose(x, ls.ls_qr(op.columns(S), y), atol=1e-9)
    assert iters <= len(S) + 2                                  # Theorem 5


def test_cg_orthogonal_case_one_step():
    # M = N: A is orthogonal, A_S^T A_S = I has a single eigenvalue -> CG ends in one step.
    op = oracle.Operator(256, 256, 9)
    S = np.arange(0, 256, 7)
    y = np.random.default_rng(1).standard_normal(256)
    x, iters, _ = ls.cg_alg1(op, S, op.apply_t(y)[S], tol=1e-12, maxit=50)
    assert iters == 1
    assert np.allclose(x, op.columns(S).T @ y, atol=1e-12)


def test_cg_warm_start_same_solution():
    op, S, y = _problem()
    b = op.apply_t(y)[S]
    x0 = np.random.default_rng(2).standard_normal(len(S))
    xw, _, _ = ls.cg_alg1(op, S, b, tol=1e-12, maxit=500, x0=x0)
    assert np.allclose(xw, ls.ls_qr(op.columns(S), y), atol=1e-9)


# ---------------------------------------------------------------- OMP (Sec. II, Algorithm 1)
def test_omp_residual_orthogonal_and_monotone():
    p = synth.workload(1)
    op = oracle.Operator(1024, 256, p.op_seed)
    s = synth.sparse_gaussian(1024, 20, 5)
    y = op.apply(s)
    norms = []

    def check(i, S, sS, r):
        assert np.abs(op.columns(S).T @ r).max() < 1e-10       # A_S^T r_i = 0
        norms.append(np.linalg.norm(r))

    greedy.omp(op, y, 20, on_step=check)
    assert np.all(np.diff(norms) <= 1e-12)


def test_omp_exact_recovery_workload1():
    # M = 1024 >> K log(N/K) = 64 ln 64 ~ 266: noiseless OMP must return the signal itself.
    p = synth.workload(1)
    op = oracle.Operator(p.N, p.M, p.op_seed)
    s = p.signal()
    res = greedy.omp(op, op.apply(s), p.K)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.abs(res["s"] - s).max() < 1e-9


def _brute_l0(op, y, kmax):
    """All supports of size <= kmax with zero residual (noiseless), smallest size first."""
    for k in range(1, kmax + 1):
        hits = []
        for S in itertools.combinations(range(op.N), k):
            S = np.array(S)
            AS = op.columns(S)
            r = y - AS @ np.linalg.lstsq(AS, y, rcond=None)[0]
            if np.linalg.norm(r) < 1e-9 * max(1.0, np.linalg.norm(y)):
                hits.append(S)
        if hits:
            return hits
    return []


def test_brute_force_l0_n16():
    """N = 16, M = 8, K <= 2: enumerate every support of size <= 2.  Where the zero-residual
    support is unique, any decoder output with zero residual must be exactly that support."""
    exercised = 0
    for seed in range(6):
        op = oracle.Operator(16, 8, 100 + seed, fast=False)
        K = 1 + seed % 2
        g = np.random.default_rng(seed)
        s = np.zeros(16)
        s[g.choice(16, K, replace=False)] = g.standard_normal(K) + np.sign(g.standard_normal(K))
        y = op.apply(s)
        hits = _brute_l0(op, y, 2)
        assert len(hits) >= 1
        if len(hits) != 1:
            continue
        truth = hits[0]
        assert np.array_equal(truth, np.flatnonzero(s))
        for algo in ("omp", "sp", "ompr"):
            res = greedy.recover(op, y, K, algo)
            if res["resid"] < 1e-9:
                assert np.array_equal(res["S"], truth), algo
                exercised += 1
    assert exercised >= 12


def test_sp_and_ompr_recover_truth_noiseless():
    N, M, K = 2048, 512, 40
    op = oracle.Operator(N, M, 21)
    s = synth.sparse_gaussian(N, K, 22)
    y = op.apply(s)
    for algo in ("sp", "ompr"):
        res = greedy.recover(op, y, K, algo)
        assert np.array_equal(res["S"], np.flatnonzero(s)), algo
        assert np.abs(res["s"] - s).max() < 1e-9, algo


def test_cosamp_recovers_truth_noiseless():
    N, M, K = 2048, 512, 40                  # 3K <= M
    op = oracle.Operator(N, M, 21)
    s = synth.sparse_gaussian(N, K, 22)
    res = greedy.cosamp(op, op.apply(s), K)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.abs(res["s"] - s).max() < 1e-9


def test_cosamp_orthonormal_operator_and_2k_merge_finish_in_one_round():
    """Two closed-form cases of the first CoSaMP round on noiseless data: (1) M = N makes A
    orthonormal, so A^T y = s and LS(T) = s on any T containing the support; (2) a signal whose
    support lies within the 2K largest |A^T y| but not within the K largest: the 2K merge puts the
    whole support into T, so LS(T) = s exactly after the first round (a K merge could not).
    Either way the first round returns s and the second sees the same support and stops."""
    opf = oracle.Operator(256, 256, 62)
    s = synth.sparse_gaussian(256, 12, 5)
    res = greedy.cosamp(opf, opf.apply(s), 12)
    assert res["iters"] == 2 and np.abs(res["s"] - s).max() < 1e-12
    N, M, K = 1024, 256, 10
    op = oracle.Operator(N, M, 61)
    for seed in range(1000, 1200):
        s = synth.sparse_gaussian(N, K, seed)
        c = np.abs(op.apply_t(op.apply(s)))
        order = np.lexsort((np.arange(N), -c))
        sup = set(np.flatnonzero(s).tolist())
        if sup <= set(order[:2 * K].tolist()) and not sup <= set(order[:K].tolist()):
            break
    else:
        pytest.fail("no signal with its support between the K and 2K largest correlations")
    res = greedy.cosamp(op, op.apply(s), K)
    assert res["iters"] == 2 and np.abs(res["s"] - s).max() < 1e-12


def test_cosamp_noisy_support_and_noise_level_error():
    N, M, K = 1 << 13, 1 << 11, 160
    p = synth.Problem(N, M, K, "cosamp", 31, 32, 33, 1e-3)
    op = oracle.Operator(N, M, p.op_seed)
    s = p.signal()
    res = greedy.cosamp(op, p.add_noise(op.apply(s)), K)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.linalg.norm(res["s"] - s) < 1e-2 * np.linalg.norm(s)


def test_sp_noisy_support_and_noise_level_error():
    N, M, K = 1 << 13, 1 << 11, 160
    p = synth.Problem(N, M, K, "sp", 31, 32, 33, 1e-3)
    op = oracle.Operator(N, M, p.op_seed)
    s = p.signal()
    y = p.add_noise(op.apply(s))
    res = greedy.sp(op, y, K)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.linalg.norm(res["s"] - s) < 1e-2 * np.linalg.norm(s)


def test_ompr_final_state_has_no_improving_swap():
    N, M, K = 1024, 256, 30
    op = oracle.Operator(N, M, 41)
    s = synth.power_law(N, K, 42)
    y = op.apply(s)
    res = greedy.ompr(op, y, K, T_max=200)
    S = res["S"]
    z = op.apply_t(y - op.apply(res["s"]))
    z[S] += res["s"][S]
    out = np.ones(N, bool)
    out[S] = False
    assert res["iters"] < 200                      # it stopped on its own rule, not on the cap
    assert np.abs(z[out]).max() <= np.abs(z[S]).min()


# ---------------------------------------------------------------- adjoint of the LS step
def test_adjoint_central_difference_exact():
    N, M, k = 1024, 256, 24
    op = oracle.Operator(N, M, 51)
    g = np.random.default_rng(52)
    S = np.sort(g.choice(N, k, replace=False))
    s_true = g.standard_normal(k)
    y = op.apply_support(S, s_true) + 0.05 * g.standard_normal(M)
    L0, grad = adjoint.loss_grad_y(op, S, y, s_true)
    eps = 1e-3
    for v in list(g.standard_normal((8, M))) + list(np.eye(M)[:8]):
        Lp, _ = adjoint.loss_grad_y(op, S, y + eps * v, s_true)
        Lm, _ = adjoint.loss_grad_y(op, S, y - eps * v, s_true)
        fd = (Lp - Lm) / (2 * eps)                               # exact for a quadratic L
        assert abs(fd - v @ grad) <= 1e-10 * max(1.0, abs(fd))


def test_adjoint_cg_route_matches_pinv():
    N, M, k = 1024, 256, 24
    op = oracle.Operator(N, M, 53)
    g = np.random.default_rng(54)
    S = np.sort(g.choice(N, k, replace=False))
    cot = g.standard_normal(k)
    dense = np.linalg.pinv(op.columns(S)).T @ cot               # (A_S^+)^T g
    assert np.allclose(adjoint.ls_backward(op, S, cot), dense, atol=1e-10)
    assert np.allclose(adjoint.ls_backward_cg(op, S, cot), dense, atol=1e-9)


# ------------------------------------------------------------------ OMPR(l), l > 1
def test_ompr_l_recovers_noiseless_and_ends_at_a_fixed_point():
    """OMPR(l) recovers a noiseless K-sparse signal at M >> K log(N/K), and its final support is
    a fixed point of the OMPR(l) step (recomputing z there selects the same S)."""
    N, M, K = 512, 160, 12
    op = oracle.Operator(N, M, 21)
    s = synth.sparse_gaussian(N, K, 22)
    y = op.apply(s)
    out = greedy.ompr(op, y, K, l=4)
    assert np.array_equal(out["S"], np.flatnonzero(s))
    assert np.linalg.norm(out["s"] - s) <= 1e-9 * np.linalg.norm(s)
    S = out["S"]
    z = op.apply_t(y - op.apply(out["s"]))
    z[S] += out["s"][S]
    a = np.abs(z)
    inside = np.zeros(N, dtype=bool)
    inside[S] = True
    J, _ = greedy.topk_lowest(a, ~inside, 4)
    union = inside.copy()
    union[J] = True
    S2, _ = greedy.topk_lowest(a, union, K)
    assert np.array_equal(S2, S)


def test_ompr_l_fixes_several_wrong_indices_per_round():
    """Starting from topK|A^T y| with several wrong indices, OMPR(l) with l = K needs fewer
    rounds than single-swap OMPR on the same input, and both end at the true support."""
    N, M, K = 1024, 256, 40
    op = oracle.Operator(N, M, 31)
    s = synth.sparse_gaussian(N, K, 32)
    y = op.apply(s)
    one = greedy.ompr(op, y, K, T_max=400)
    many = greedy.ompr(op, y, K, T_max=400, l=K)
    truth = np.flatnonzero(s)
    assert np.array_equal(one["S"], truth) and np.array_equal(many["S"], truth)
    assert many["iters"] < one["iters"]


# ------------------------------------------------------------ permutation randomiser R
def test_perm_is_a_permutation_and_the_operator_is_the_permuted_dct():
    """Sec. III-A's R as a uniform random permutation: A = P_Omega C_N Pi equals the orthonormal
    DCT matrix (scipy) restricted to Omega, with its columns permuted by perm."""
    N, M = 256, 70
    op = oracle.Operator(N, M, 5, randomizer="perm")
    assert np.array_equal(np.sort(op.perm), np.arange(N))
    assert not np.array_equal(op.perm, np.arange(N))
    C = sfft.dct(np.eye(N), axis=0, norm="ortho")
    want = np.empty((M, N))
    want[:, op.perm] = C[op.omega, :]          # column perm[n] of A is column n of C
    assert np.allclose(op.dense(), want, atol=1e-12)
    g = np.random.default_rng(1)
    x = g.standard_normal(N)
    u = g.standard_normal(M)
    assert np.allclose(op.apply(x), want @ x, atol=1e-12)
    assert np.allclose(op.apply_t(u), want.T @ u, atol=1e-12)
    assert np.allclose(op.apply(op.apply_t(u)), u, atol=1e-12)   # A A^T = I_M


def test_perm_operator_recovers_noiseless_sparse():
    N, M, K = 1024, 256, 20
    op = oracle.Operator(N, M, 9, randomizer="perm")
    s = synth.sparse_gaussian(N, K, 10)
    for algo in ("omp", "sp", "ompr"):
        out = greedy.recover(op, op.apply(s), K, algo)
        assert np.array_equal(out["S"], np.flatnonzero(s)), algo
        assert np.linalg.norm(out["s"] - s) <= 1e-9 * np.linalg.norm(s)



# ------------------------------------------------------------ sparsifying basis Psi
def test_psi_dct_with_no_randomiser_is_row_sampling():
    """Closed form: with R = I and Psi = C_N^T, A = P_Omega C_N C_N^T = P_Omega, so A s = s[Omega]
    and A^T u scatters u onto Omega."""
    N, M = 256, 64
    op = oracle.Operator(N, M, 3, randomizer="none", psi="dct")
    s = np.random.default_rng(0).standard_normal(N)
    assert np.abs(op.apply(s) - s[op.omega]).max() < 1e-12
    u = np.random.default_rng(1).standard_normal(M)
    want = np.zeros(N)
    want[op.omega] = u
    assert np.abs(op.apply_t(u) - want).max() < 1e-12


def test_psi_dct2d_basis_is_scipy_idctn():
    """The separable basis: Psi vec(S) = vec(idctn(S)) (scipy, orthonormal), row-major."""
    import scipy.fft as sfft
    op = oracle.Operator(512, 128, 4, psi=("dct2d", 16, 32))
    S = np.random.default_rng(2).standard_normal((16, 32))
    assert np.abs(op._psi(S.ravel()) - sfft.idctn(S, norm="ortho").ravel()).max() < 1e-12
    assert np.abs(op._psi_t(S.ravel()) - sfft.dctn(S, norm="ortho").ravel()).max() < 1e-12


@pytest.mark.parametrize("psi", ["dct", ("dct2d", 16, 32)])
def test_psi_operator_keeps_orthonormal_rows_and_columns_agree(psi):
    N, M = 512, 128
    op = oracle.Operator(N, M, 5, psi=psi)
    A = op.dense()
    assert np.abs(A @ A.T - np.eye(M)).max() < 1e-12
    x = np.random.default_rng(3).standard_normal(N)
    assert np.abs(A @ x - op.apply(x)).max() < 1e-12
    u = np.random.default_rng(4).standard_normal(M)
    assert np.abs(A.T @ u - op.apply_t(u)).max() < 1e-12


@pytest.mark.parametrize("algo", ["omp", "sp", "cosamp"])
def test_psi_dct_sparse_signal_recovered_exactly(algo):
    """An image sparse in the 2-D DCT basis (the coefficients are the unknown), noiseless."""
    N, M, K = 1024, 256, 20
    op = oracle.Operator(N, M, 6, psi=("dct2d", 32, 32))
    s = synth.sparse_gaussian(N, K, 7)
    res = greedy.recover(op, op.apply(s), K, algo)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.abs(res["s"] - s).max() < 1e-9



# -------------------------------------------------------------- any N (not only 2^k)
@pytest.mark.parametrize("N", [1000, 999, 24])
def test_operator_at_non_power_of_two_n(N):
    """The oracle takes any N (the GPU path takes powers of two): A = P_Omega C_N diag(d) equals
    scipy's orthonormal DCT-II on the rows Omega, and A A^T = I_M."""
    import scipy.fft as sfft
    M = N // 4
    op = oracle.Operator(N, M, 9)
    C = sfft.dct(np.eye(N), norm="ortho", axis=0)
    A = C[op.omega] * op.d[None, :]
    assert np.abs(op.dense() - A).max() < 1e-12
    assert np.abs(A @ A.T - np.eye(M)).max() < 1e-12
    x = np.random.default_rng(N).standard_normal(N)
    assert np.abs(op.apply(x) - A @ x).max() < 1e-12


def test_sp_exact_recovery_at_non_power_of_two_n():
    N, M, K = 1000, 250, 12
    op = oracle.Operator(N, M, 10)
    s = synth.sparse_gaussian(N, K, 11)
    res = greedy.sp(op, op.apply(s), K)
    assert np.array_equal(res["S"], np.flatnonzero(s))
    assert np.abs(res["s"] - s).max() < 1e-9
