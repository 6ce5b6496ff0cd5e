"""CPU checks of the selection-parity harness (tests/replay.py): a trace in the library's
documented layout, written here from an oracle run, must replay cleanly; a wrong choice at a
clear margin must fail; another member of a near-tied set must be accepted and followed."""
import numpy as np
import pytest

import oracle
from oracle import greedy
from paper_1509_03979_gb300 import synth
from oracle import replay

CODES = {"argmax": 1, "argmin": 2, "topk": 3, "stop": 4, "swap": 5}


class _Writer(greedy.OwnChoice):
    """Records the oracle's own choices in the trace layout of cs_op_set_trace."""

    def __init__(self, N, override=None):
        self.W = (N + 31) // 32
        self.words = [0, 0, 0, self.W]
        self.n = 0
        self.override = override or {}

    def _rec(self, kind, mu, aux, payload=()):
        self.words += [CODES[kind], len(payload), int(np.array([mu], np.float32).view(np.uint32)[0]), aux]
        self.words += list(payload)
        self.n += 1

    def select(self, kind, own, mu, a, allowed, values="corr"):
        own = self.override.get(self.n, own)
        if kind == "topk":
            bits = np.zeros(self.W * 32, dtype=np.uint8)
            bits[np.asarray(own)] = 1
            payload = np.packbits(bits, bitorder="little").view(np.uint32).tolist()
            self._rec(kind, mu, len(own), payload)
        else:
            self._rec(kind, mu, int(own))
        return own

    def decide(self, kind, own, mu, vals=None):
        self._rec(kind, mu, int(bool(own)))
        return own

    def trace(self):
        t = np.array(self.words, dtype=np.int64)
        t[0], t[1] = len(t), self.n
        return t.astype(np.uint32).view(np.int32)


def _run(algo, N=1024, M=300, K=20, noise=1e-3, override=None, **kw):
    op = oracle.Operator(N, M, 3)
    p = synth.Problem(N, M, K, algo, 3, 4, 5, noise)
    y = p.add_noise(op.apply(p.signal()))
    w = _Writer(N, override)
    res = greedy.recover(op, y, K, algo, policy=w, **kw)
    return op, y, res, w.trace()


@pytest.mark.parametrize("algo,kw", [("omp", {}), ("sp", {}), ("ompr", {}), ("ompr", {"l": 5}), ("cosamp", {})])
def test_own_trace_replays_exactly(algo, kw):
    op, y, res, tr = _run(algo, **kw)
    rep, ref = replay.check_recovery(op, y, 20, algo, tr, res["s"], res["S"], 1e-12, **kw)
    assert rep["diverged"] == [] and rep["max_margin_gap"] < 1e-6
    assert len(replay.parse_trace(tr)) == len(res["trace"])


def test_wrong_choice_at_a_clear_margin_fails():
    op, y, res, tr = _run("omp")
    recs = replay.parse_trace(tr)
    first = [i for i, r in enumerate(recs) if r["mu"] > 0.05][0]
    # rewrite that record's index to another candidate
    off = replay.HEADER + 4 * first
    bad = tr.copy()
    bad[off + 3] = (int(bad[off + 3]) + 1) % op.N
    with pytest.raises(AssertionError):
        replay.check_recovery(op, y, 20, "omp", bad, res["s"], res["S"], 1e-6)


def test_other_member_of_a_tie_is_followed():
    # orthonormal operator, two exactly tied magnitudes: the second member may be taken first
    N = 256
    op = oracle.Operator(N, N, 77)
    s = np.zeros(N)
    s[[5, 42, 79]] = [3.0, -3.0, 1.0]
    y = op.apply(s)
    own = greedy.omp(op, y, 3)
    other = 42 if own["trace"] and int(np.argmax(np.abs(op.apply_t(y)))) == 5 else 5
    w = _Writer(N, override={0: other})
    res = greedy.omp(op, y, 3, policy=w)
    rep, ref = replay.check_recovery(op, y, 3, "omp", w.trace(), res["s"], res["S"], 1e-12)
    assert rep["diverged"] and rep["diverged"][0][1] == "argmax"


def test_overflowed_trace_is_rejected():
    op, y, res, tr = _run("sp")
    bad = tr.copy()
    bad[2] = 1
    with pytest.raises(AssertionError):
        replay.parse_trace(bad)
