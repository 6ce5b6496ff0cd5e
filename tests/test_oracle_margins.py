"""Pins of the oracle's selection margins, near-tie counts, selection policies and its growing
Cholesky LS (CPU only).

The margins decide where the GPU decoders must agree with the oracle exactly (margin above
1e-3) and where a different member of a near-tied set is accepted, so they are pinned on
hand-built vectors with known gaps (exact ties, a gap of exactly 1e-3, the K boundary of
top-K) and, inside the decoders, against closed forms: with M = N the operator is orthonormal,
A^T A = I, so OMP's i-th correlation is the true signal minus what has been found and its i-th
argmax margin is the i-th relative gap of the sorted |s|.
"""
import numpy as np
import pytest

import oracle
from oracle import greedy, ls


# ------------------------------------------------------------------- hand-built vectors
def test_argmax_exact_tie_takes_the_lowest_index_with_margin_zero():
    t, mu = greedy._argmax_lowest(np.array([1.0, 3.0, 2.0, 3.0]), np.ones(4, bool))
    assert (t, mu) == (1, 0.0)


def test_argmax_ignores_excluded_entries():
    allowed = np.array([False, True, True, True])
    t, mu = greedy._argmax_lowest(np.array([9.0, 3.0, 2.0, 3.0]), allowed)
    assert (t, mu) == (1, 0.0)
    t, mu = greedy._argmax_lowest(np.array([9.0, 4.0, 2.0, 3.0]), allowed)
    assert t == 1 and mu == pytest.approx(0.25, abs=0)


def test_argmax_margin_uses_the_winner_as_denominator():
    t, mu = greedy._argmax_lowest(np.array([2.0, 4.0]), np.ones(2, bool))
    assert t == 1 and mu == 0.5          # (4 - 2) / 4, not (4 - 2) / 2


def test_argmax_gap_of_exactly_1e3_is_a_near_tie():
    t, mu = greedy._argmax_lowest(np.array([999.0, 1000.0, 0.5]), np.ones(3, bool))
    assert t == 1 and mu == 1e-3 and mu <= greedy.NEAR_TIE
    # just inside and just outside the band, with exactly representable gaps
    _, mu_in = greedy._argmax_lowest(np.array([1.0, 1.0 - 2.0 ** -10]), np.ones(2, bool))
    _, mu_out = greedy._argmax_lowest(np.array([1.0, 1.0 - 2.0 ** -9]), np.ones(2, bool))
    assert mu_in == 2.0 ** -10 and mu_in <= greedy.NEAR_TIE
    assert mu_out == 2.0 ** -9 and mu_out > greedy.NEAR_TIE


def test_argmax_single_candidate_has_margin_one():
    allowed = np.array([False, False, True])
    assert greedy._argmax_lowest(np.array([5.0, 6.0, 0.25]), allowed) == (2, 1.0)


def test_argmin_ties_and_margin():
    assert greedy._argmin_lowest(np.array([5.0, 2.0, 3.0, 2.0]), np.ones(4, bool)) == (1, 0.0)
    t, mu = greedy._argmin_lowest(np.array([4.0, 2.0, 3.0]), np.ones(3, bool))
    assert t == 1 and mu == pytest.approx(1.0 / 3.0, rel=1e-15)     # (3 - 2) / 3
    assert greedy._argmin_lowest(np.array([4.0, 2.0]), np.array([True, False])) == (0, 1.0)


@pytest.mark.parametrize("K,want,mu", [
    (1, [0], 0.2),                  # (5 - 4) / 5
    (2, [0, 1], 0.25),              # (4 - 3) / 4
    (3, [0, 1, 2], 0.0),            # tie 3 = 3 at the boundary: index 2 wins, margin 0
    (4, [0, 1, 2, 3], 2.0 / 3.0),   # (3 - 1) / 3
    (5, [0, 1, 2, 3, 4], 1.0),      # every candidate taken: a_(K+1) = 0
])
def test_topk_boundary_and_margin(K, want, mu):
    pick, m = greedy.topk_lowest(np.array([5.0, 4.0, 3.0, 3.0, 1.0]), np.ones(5, bool), K)
    assert pick.tolist() == want and m == pytest.approx(mu, rel=1e-15, abs=0)


def test_topk_over_a_restricted_set_and_a_tie_resolved_by_index():
    a = np.array([7.0, 2.0, 6.0, 2.0, 9.0, 2.0])
    allowed = np.array([True, True, True, True, False, True])
    pick, mu = greedy.topk_lowest(a, allowed, 3)
    assert pick.tolist() == [0, 1, 2] and mu == 0.0        # 2 = 2: the lowest index (1) wins
    pick, mu = greedy.topk_lowest(a, allowed, 2)
    assert pick.tolist() == [0, 2] and mu == pytest.approx(4.0 / 6.0, rel=1e-15)


def test_finish_counts_near_ties_at_and_below_the_threshold():
    op = oracle.Operator(16, 8, 1)
    trace = [("argmax", 0.5), ("topk", 1e-3), ("topk", 2e-3), ("stop", 0.0), ("swap", 1.0)]
    res = greedy._finish(op, np.zeros(8), np.array([3]), np.array([0.0]), 1, trace)
    assert res["near_ties"] == 2 and res["min_margin"] == 0.0
    res = greedy._finish(op, np.zeros(8), np.array([3]), np.array([0.0]), 1, [("argmax", 0.5)])
    assert res["near_ties"] == 0 and res["min_margin"] == 0.5
    res = greedy._finish(op, np.zeros(8), np.array([3]), np.array([0.0]), 0, [])
    assert res["near_ties"] == 0 and res["min_margin"] == 1.0


# ------------------------------------------------------------ margins inside the decoders
def _orthonormal_problem(mags):
    """M = N: A = C_N diag(d) is orthonormal, so A^T A = I.  s has the given magnitudes (in this
    order of size) at scattered positions with alternating signs."""
    N = 256
    op = oracle.Operator(N, N, 77)
    pos = (np.arange(len(mags)) * 37 + 5) % N
    s = np.zeros(N)
    s[pos] = np.asarray(mags) * np.where(np.arange(len(mags)) % 2 == 0, 1.0, -1.0)
    return op, s, pos


def test_omp_margins_are_the_gaps_of_the_sorted_signal_on_an_orthonormal_operator():
    mags = [10.0, 9.995, 5.0, 4.0, 3.999, 1.0]
    op, s, pos = _orthonormal_problem(mags)
    K = len(mags)
    res = greedy.omp(op, op.apply(s), K)
    want = [(mags[i] - (mags[i + 1] if i + 1 < K else 0.0)) / mags[i] for i in range(K)]
    got = [m for _, m in res["trace"]]
    assert np.allclose(got, want, rtol=0, atol=1e-9)
    assert res["near_ties"] == 2                        # 10 vs 9.995 and 4 vs 3.999
    assert res["min_margin"] == pytest.approx(min(want), abs=1e-9)
    assert np.array_equal(res["S"], np.sort(pos))


def test_ompr_initial_topk_argmin_and_swap_margins_in_closed_form():
    # orthonormal operator: the initial top-K is the true support, LS is exact, so z = s on S
    # and 0 outside; argmax outside has a_j = 0, argmin inside is the smallest |s| and the swap
    # test |z_j| > |z_i| fails with margin 1
    mags = [8.0, 6.0, 5.0, 4.5]
    op, s, pos = _orthonormal_problem(mags)
    res = greedy.ompr(op, op.apply(s), len(mags))
    kinds = [k for k, _ in res["trace"]]
    assert kinds == ["topk", "argmax", "argmin", "swap"] and res["iters"] == 0
    m = dict(res["trace"])
    assert m["topk"] == pytest.approx(1.0, abs=1e-12)
    assert m["argmin"] == pytest.approx((5.0 - 4.5) / 5.0, abs=1e-9)
    assert m["swap"] == pytest.approx(1.0, abs=1e-12)


def test_sp_records_its_residual_stop_test():
    mags = [3.0, 2.0, 1.0]
    op, s, pos = _orthonormal_problem(mags)
    res = greedy.sp(op, op.apply(s), 3)
    kinds = [k for k, _ in res["trace"]]
    assert kinds == ["topk", "topk", "topk", "stop"]
    assert dict(res["trace"])["stop"] == 1.0           # S' = S: decided by set equality


# ------------------------------------------------------------------------- policies
class _Recorder(greedy.OwnChoice):
    def __init__(self):
        self.events = []

    def select(self, kind, own, mu, a, allowed, values="corr"):
        self.events.append(kind)
        return own

    def decide(self, kind, own, mu, vals=None):
        self.events.append(kind)
        return own


@pytest.mark.parametrize("algo,kw,head,body", [
    ("sp", {}, ["topk"], ["topk", "topk", "stop"]),
    ("cosamp", {}, [], ["topk", "topk", "stop"]),
    ("ompr", {}, ["topk"], ["argmax", "argmin", "swap"]),
    ("ompr", {"l": 4}, ["topk"], ["topk", "topk", "stop"]),
])
def test_policy_sees_every_selection_in_decoder_order(algo, kw, head, body):
    op = oracle.Operator(512, 160, 5)
    from paper_1509_03979_gb300 import synth
    s = synth.sparse_gaussian(512, 12, 9)
    rec = _Recorder()
    res = greedy.recover(op, op.apply(s), 12, algo, policy=rec, **kw)
    ev = rec.events
    assert ev[:len(head)] == head
    tail = ev[len(head):]
    assert len(tail) % len(body) == 0 and tail == body * (len(tail) // len(body))
    assert [k for k, _ in res["trace"]] == ev


def test_forced_sequence_replays_omp_and_can_take_another_member_of_a_tie():
    mags = [10.0, 10.0, 4.0, 2.0]          # a tie between the two largest
    op, s, pos = _orthonormal_problem(mags)
    y = op.apply(s)
    rec = []

    class Log(greedy.OwnChoice):
        def select(self, kind, own, mu, a, allowed, values="corr"):
            rec.append(own)
            return own
    own = greedy.omp(op, y, 4, policy=Log())
    assert own["trace"][0][1] <= 1e-12 and own["near_ties"] >= 1
    assert set(rec[:2]) == {int(pos[0]), int(pos[1])}
    again = greedy.omp(op, y, 4, replay=rec)
    other = greedy.omp(op, y, 4, replay=[rec[1], rec[0]] + rec[2:])
    for r in (again, other):
        assert np.array_equal(r["S"], own["S"]) and np.abs(r["s"] - own["s"]).max() < 1e-12


# -------------------------------------------------------------------- growing Cholesky
def test_growing_cholesky_equals_qr_for_any_insertion_order():
    op = oracle.Operator(1024, 256, 13)
    g = np.random.default_rng(3)
    S = g.choice(1024, 40, replace=False)
    y = g.standard_normal(256)
    ch = ls.GrowingCholesky(op, y, capacity=4)         # forces the storage to grow
    for t in S:
        ch.add(t)
    Ss, x = ch.solve()
    assert np.array_equal(Ss, np.sort(S))
    want = ls.ls_qr(op.columns(Ss), y)
    assert np.abs(x - want).max() <= 1e-10 * np.abs(want).max()


def test_omp_with_the_growing_factor_matches_qr_omp():
    from paper_1509_03979_gb300 import synth
    op = oracle.Operator(1024, 256, 21)
    s = synth.sparse_gaussian(1024, 40, 22)
    y = op.apply(s) + 1e-3 * synth.normals(23, 256)
    a = greedy.omp(op, y, 40, ls_method="qr")
    b = greedy.omp(op, y, 40, ls_method="grow")
    assert np.array_equal(a["S"], b["S"])
    assert np.abs(a["s"] - b["s"]).max() <= 1e-10
    assert np.allclose([m for _, m in a["trace"]], [m for _, m in b["trace"]], rtol=0, atol=1e-10)


def test_warm_started_cg_reaches_the_closed_form():
    op = oracle.Operator(2048, 512, 31)
    g = np.random.default_rng(4)
    S = np.sort(g.choice(2048, 60, replace=False))
    y = g.standard_normal(512)
    want = ls.ls_qr(op.columns(S), y)
    x0 = want + 0.1 * g.standard_normal(60)
    got = ls.ls_cg(op, S, y, x0=x0)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
