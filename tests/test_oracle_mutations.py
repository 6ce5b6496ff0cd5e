"""Planted mistakes in the FP64 oracle (CPU only): each test patches one plausible error into
an oracle function -- a wrong weight, a dropped or flipped sign, a transposed index, a skipped
reordering, an off-by-one, an inverted recurrence -- and checks that the pins of
test_oracle_pins.py (or the host-draw cross-check) catch it.  The oracle itself is never
changed on disk; monkeypatch restores it after every test.  (Letting OMP re-select an index
already in S is not such a mistake: the residual is orthogonal to A_S after each LS, so the
argmax never lands in S and the pins rightly see no difference.)"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle import adjoint, dct, greedy, ls, rng
from tests import test_oracle_margins as margins
from tests import test_oracle_pins as pins


def caught(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


# ---------------------------------------------------------------------------- DCT
def test_wrong_dc_weight_is_caught(monkeypatch):
    monkeypatch.setattr(dct, "weights", lambda N: np.full(N, np.sqrt(2.0 / N)))
    caught(pins.test_dct_naive_matches_scipy, 64)
    caught(pins.test_dct_fast_matches_scipy, 64)


def test_flipped_phase_sign_is_caught(monkeypatch):
    def bad(x):
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[-1]
        v = np.concatenate([x[..., 0::2], x[..., 1::2][..., ::-1]], axis=-1)
        V = np.fft.fft(v, axis=-1)
        k = np.arange(N)
        return dct.weights(N) * np.real(np.exp(+1j * np.pi * k / (2.0 * N)) * V)
    monkeypatch.setattr(dct, "dct2_fast", bad)
    caught(pins.test_dct_fast_matches_scipy, 64)


def test_missing_reversal_in_the_reordering_is_caught(monkeypatch):
    def bad(x):
        x = np.asarray(x, dtype=np.float64)
        N = x.shape[-1]
        v = np.concatenate([x[..., 0::2], x[..., 1::2]], axis=-1)
        V = np.fft.fft(v, axis=-1)
        k = np.arange(N)
        return dct.weights(N) * np.real(np.exp(-1j * np.pi * k / (2.0 * N)) * V)
    monkeypatch.setattr(dct, "dct2_fast", bad)
    caught(pins.test_dct_fast_matches_scipy, 64)


# ------------------------------------------------------------------------ operator
def test_dropped_sign_flip_in_the_transpose_is_caught(monkeypatch):
    def bad(self, u):
        u = np.asarray(u, dtype=np.float64)
        full = np.zeros(u.shape[:-1] + (self.N,))
        full[..., self.omega] = u
        return self._ct(full)                      # d forgotten
    monkeypatch.setattr(oracle.Operator, "apply_t", bad)
    caught(pins.test_operator_apply_matches_dense, True)


def test_transposed_cosine_index_is_caught(monkeypatch):
    def bad(self, S):
        S = np.asarray(S, dtype=np.int64)
        k = self.omega[:, None].astype(np.float64)
        j = S[None, :].astype(np.float64)
        w = dct.weights(self.N)[self.omega][:, None]
        return self.d[S][None, :] * w * np.cos(np.pi * (2.0 * k + 1.0) * j / (2.0 * self.N))
    monkeypatch.setattr(oracle.Operator, "columns", bad)
    caught(pins.test_operator_apply_matches_dense, True)


# ----------------------------------------------------------------------------- CG
def _cg(update_sign=-1.0, beta_inverted=False):
    def cg(op, S, b, tol, maxit, x0=None, absolute=False):
        S = np.asarray(S, dtype=np.int64)
        x = np.zeros(len(S)) if x0 is None else np.array(x0, dtype=np.float64)
        r = b - ls.gram_apply(op, S, x) if x0 is not None else np.array(b, dtype=np.float64)
        d = r.copy()
        rr = float(r @ r)
        stop = tol if absolute else tol * float(np.sqrt(b @ b))
        j = 0
        while np.sqrt(rr) > stop and j < maxit:
            Hd = ls.gram_apply(op, S, d)
            alpha = rr / float(d @ Hd)
            x = x + alpha * d
            r = r + update_sign * alpha * Hd
            rr_new = float(r @ r)
            beta = rr / rr_new if beta_inverted else rr_new / rr
            d = r + beta * d
            rr = rr_new
            j += 1
        return x, j, float(np.sqrt(rr))
    return cg


def test_wrong_residual_sign_in_cg_is_caught(monkeypatch):
    monkeypatch.setattr(ls, "cg_alg1", _cg(update_sign=+1.0))
    caught(pins.test_theorem2_cg_matches_closed_form_and_theorem5_bound)


def test_inverted_beta_in_cg_is_caught(monkeypatch):
    monkeypatch.setattr(ls, "cg_alg1", _cg(beta_inverted=True))
    caught(pins.test_theorem2_cg_matches_closed_form_and_theorem5_bound)


# ------------------------------------------------------------------------ decoders
def test_argmax_off_by_one_is_caught(monkeypatch):
    """The argmax takes the runner-up (order[1] for order[0])."""
    def bad(a, allowed):
        idx = np.flatnonzero(allowed)
        vals = a[idx]
        order = np.lexsort((idx, -vals))
        t = int(idx[order[1]]) if len(order) > 1 else int(idx[order[0]])
        return t, 0.5
    monkeypatch.setattr(greedy, "_argmax_lowest", bad)
    caught(pins.test_omp_exact_recovery_workload1)


def test_topk_taking_the_smallest_is_caught(monkeypatch):
    orig = greedy.topk_lowest
    monkeypatch.setattr(greedy, "topk_lowest", lambda a, allowed, K: orig(-a, allowed, K))
    caught(pins.test_sp_and_ompr_recover_truth_noiseless)


def test_adjoint_without_the_solve_is_caught(monkeypatch):
    monkeypatch.setattr(adjoint, "ls_backward", lambda op, S, g: op.columns(S) @ np.asarray(g, dtype=np.float64))
    caught(pins.test_adjoint_cg_route_matches_pinv)


# ------------------------------------------------------------------------ draws
def test_off_by_one_in_the_omega_shuffle_is_caught(monkeypatch):
    def bad(N, M, seed):
        u = rng.stream((seed ^ rng.GAMMA) & ((1 << 64) - 1), M)
        perm = np.arange(N, dtype=np.int64)
        for i in range(M):
            span = max(N - i - 1, 1)                 # N - i - 1 instead of N - i
            j = i + int(u[i] % np.uint64(span))
            perm[i], perm[j] = perm[j], perm[i]
        return np.sort(perm[:M])
    monkeypatch.setattr(rng, "omega", bad)
    caught(pins.test_omega_uniform_inclusion)


def test_wrong_sign_salt_is_caught_by_the_host_draw_cross_check(monkeypatch):
    from paper_1509_03979_gb300 import binding, build
    build.build()
    lib = binding.lib()
    orig = rng.signs
    monkeypatch.setattr(rng, "signs", lambda N, seed: orig(N, seed ^ 1))
    N, M, seed = 4096, 1024, 0x0C5001
    d = np.zeros(N, dtype=np.int8)
    assert lib.cs_operator_draws(N, M, seed, None, d.ctypes.data_as(ctypes.c_void_p)) == 0
    assert not np.array_equal(d.astype(np.float64), rng.signs(N, seed))


def test_cosamp_merging_k_instead_of_2k_is_caught(monkeypatch):
    orig = greedy.topk_lowest

    def half(a, allowed, K):
        # the first selection of each CoSaMP round is the only one over all indices
        return orig(a, allowed, K // 2 if allowed.all() and K % 2 == 0 else K)
    monkeypatch.setattr(greedy, "topk_lowest", half)
    caught(pins.test_cosamp_orthonormal_operator_and_2k_merge_finish_in_one_round)


def test_psi_applied_as_its_transpose_is_caught(monkeypatch):
    def bad(self, s):
        s = np.asarray(s, dtype=np.float64)
        return s if self.psi is None else self._c(s)      # C_N instead of C_N^T
    monkeypatch.setattr(oracle.Operator, "_psi", bad)
    caught(pins.test_psi_dct_with_no_randomiser_is_row_sampling)


# ------------------------------------------------------------------------ margins
def test_every_margin_forced_to_zero_is_caught(monkeypatch):
    """Every selection reported as a near-tie would silently switch off every exact support
    check on the GPU side."""
    orig = greedy._finish
    monkeypatch.setattr(greedy, "_finish",
                        lambda op, y, S, sS, iters, trace: orig(op, y, S, sS, iters, [(k, 0.0) for k, _ in trace]))
    caught(margins.test_finish_counts_near_ties_at_and_below_the_threshold)
    caught(margins.test_omp_margins_are_the_gaps_of_the_sorted_signal_on_an_orthonormal_operator)


def test_argmax_margin_over_the_runner_up_is_caught(monkeypatch):
    def bad(a, allowed):
        idx = np.flatnonzero(allowed)
        vals = a[idx]
        order = np.lexsort((idx, -vals))
        a1 = float(vals[order[0]])
        a2 = float(vals[order[1]]) if len(order) > 1 else 0.0
        return int(idx[order[0]]), (a1 - a2) / a2 if a2 > 0 else 1.0    # wrong denominator
    monkeypatch.setattr(greedy, "_argmax_lowest", bad)
    caught(margins.test_argmax_margin_uses_the_winner_as_denominator)
    caught(margins.test_omp_margins_are_the_gaps_of_the_sorted_signal_on_an_orthonormal_operator)


def test_topk_margin_against_the_wrong_neighbour_is_caught(monkeypatch):
    def bad(a, allowed, K):
        idx = np.flatnonzero(allowed)
        vals = a[idx]
        order = np.lexsort((idx, -vals))
        aK = float(vals[order[K - 1]])
        aKm1 = float(vals[order[K - 2]]) if K >= 2 else aK             # a_(K-1) for a_(K+1)
        return np.sort(idx[order[:K]]), (aKm1 - aK) / aKm1 if aKm1 > 0 else 0.0
    monkeypatch.setattr(greedy, "topk_lowest", bad)
    caught(margins.test_topk_boundary_and_margin, 2, [0, 1], 0.25)


def test_ompr_that_never_stops_is_caught(monkeypatch):
    class Always(greedy.OwnChoice):
        def decide(self, kind, own, mu, vals=None):
            return True if kind == "swap" else own
    orig = greedy.ompr
    monkeypatch.setattr(greedy, "ompr", lambda *a, **k: orig(*a, **dict(k, policy=Always())))
    caught(pins.test_ompr_final_state_has_no_improving_swap)
