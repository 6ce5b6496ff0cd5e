"""Oracle greedy decoders OMP, SP, OMPR and CoSaMP in FP64 (test infrastructure only).

Each decoder alternates support detection (a correlation A^T r and a selection over |.|) with
the least-squares sub-problem on the current support (Sec. II).  The oracle solves every LS
sub-problem in closed form (QR of A_S, or for OMP's growing support the incrementally extended
Cholesky factor of A_S^T A_S) or, when A_S would not fit, by FP64 CG to 1e-13 relative -- the
value the paper's CG approximates (Theorems 1-2).

  * OMP: Sec. II steps 1-4 and the outer loop of Algorithm 1 (exactly K iterations).
  * SP: Subspace Pursuit (Dai & Milenkovic 2009), which the paper only cites.  Reading used:
      S <- topK|A^T y|; s <- LS(S); r <- y - A s; then repeat: S~ = S u topK_{j not in S}|A^T r|,
      u <- LS(S~), S' <- topK_{j in S~}|u_j|, s' <- LS(S'), r' <- y - A s'; stop and keep
      (s, S) if S' = S or ||r'|| >= ||r||, else accept (S', s', r').  At most L_max rounds.
  * OMPR: OMP with Replacement (Jain, Tewari & Dhillon 2011), also only cited.  Reading used
      (step eta = 1, one replacement per iteration): S <- topK|A^T y|; s <- LS(S); then for at
      most T_max rounds: z = s + A^T r, j = argmax_{not in S}|z_j|, i = argmin_{in S}|z_i|;
      stop if |z_j| <= |z_i|; else S <- S - {i} + {j}, s <- LS(S), r <- y - A s.
      OMPR(l), l > 1 replacements per round (the generalisation in the same paper): J = the l
      largest |z_j| outside S, S' = the K largest |z| over S u J; stop if S' = S, else
      S <- S', s <- LS(S), r <- y - A s.
  * CoSaMP (Needell & Tropp 2009), a relative of SP that the paper does not treat.  Reading used
      (with SP's stopping rule): S <- {}, s <- 0, r <- y; then repeat: T = S u top2K|A^T r|
      (the 2K largest over all indices), b <- LS(T), S' <- topK_{j in T}|b_j|, s' <- b on S'
      (no second LS), r' <- y - A s'; stop and keep (s, S) if S' = S or ||r'|| >= ||r||, else
      accept.  At most L_max rounds.  Needs 3K <= M.

Ties are broken towards the lowest index everywhere.  Every selection records its margin
mu = (a_(1) - a_(2)) / a_(1) (argmax), (a_(2) - a_(1)) / a_(2) (argmin) or
(a_(K) - a_(K+1)) / a_(K) (top-K), and every data-dependent stop test records one too:
|a_j - a_i| / max(a_j, a_i) for OMPR's swap test, |rho - rho'| / max(rho, rho') for the residual
test rho' >= rho of SP and CoSaMP, and 1 for a test decided by set equality (S' = S).
mu <= 1e-3 marks a near-tie, at which an FP32 decoder may legitimately choose differently.

Every selection and stop test goes through a `policy` object (default `OwnChoice`: take the
oracle's own choice).  A replaying policy can substitute another decoder's recorded choices --
the replay mode in which an FP32 trajectory that took a different member of a near-tied set is
followed, so that the rest of its run can still be compared.  A policy changes only discrete
choices, never the arithmetic.
"""
import numpy as np

from . import ls as _ls

NEAR_TIE = 1e-3


def _argmax_lowest(a, allowed):
    """Index of the largest a over `allowed` (lowest index on ties) and the selection margin
    (a_(1) - a_(2)) / a_(1), with a_(2) = 0 when only one index is allowed."""
    idx = np.flatnonzero(allowed)
    vals = a[idx]
    order = np.lexsort((idx, -vals))
    t = int(idx[order[0]])
    a1 = float(vals[order[0]])
    a2 = float(vals[order[1]]) if len(order) > 1 else 0.0
    return t, (a1 - a2) / a1 if a1 > 0 else 0.0


def _argmin_lowest(a, allowed):
    """Index of the smallest a over `allowed` (lowest index on ties) and the margin
    (a_(2) - a_(1)) / a_(2); 1 when only one index is allowed."""
    idx = np.flatnonzero(allowed)
    vals = a[idx]
    order = np.lexsort((idx, vals))
    t = int(idx[order[0]])
    a1 = float(vals[order[0]])
    a2 = float(vals[order[1]]) if len(order) > 1 else np.inf
    return t, (a2 - a1) / a2 if np.isfinite(a2) and a2 > 0 else (1.0 if a2 > a1 else 0.0)


def topk_lowest(a, allowed, K):
    """The K indices with the largest a among `allowed` (ties -> lowest index), sorted ascending,
    and the boundary margin (a_(K) - a_(K+1)) / a_(K), with a_(K+1) = 0 when all are taken."""
    idx = np.flatnonzero(allowed)
    vals = a[idx]
    order = np.lexsort((idx, -vals))
    pick = idx[order[:K]]
    aK = float(vals[order[K - 1]])
    aK1 = float(vals[order[K]]) if len(order) > K else 0.0
    mu = (aK - aK1) / aK if aK > 0 else 0.0
    return np.sort(pick), mu


def _test_margin(x, x_new):
    """Margin of the comparison x_new >= x: |x - x_new| / max(x, x_new)."""
    big = max(x, x_new)
    return abs(x - x_new) / big if big > 0 else 0.0


class OwnChoice:
    """Selection policy that keeps the oracle's own choice at every step.

    select(kind, own, mu, a, allowed, values): kind is "argmax", "argmin" or "topk"; own the
    oracle's index (argmax / argmin) or sorted index array (top-K); a the values it selected on,
    allowed the candidate mask, values what a holds: "corr" (correlations |A^T r|, or z outside
    the support) or "coef" (least-squares coefficients, or z inside the support).
    decide(kind, own, mu, vals): kind "swap" (own: True = swap; vals = (|z_i|, |z_j|, |S|)) or "stop"
    (own: True = stop; vals = (||r||, ||r'||), None when set equality decided it).  Both return
    the choice the decoder continues with."""

    def select(self, kind, own, mu, a, allowed, values="corr"):
        return own

    def decide(self, kind, own, mu, vals=None):
        return own


class ForcedSequence(OwnChoice):
    """OMP replay: the i-th argmax takes index seq[i]."""

    def __init__(self, seq):
        self.seq = list(seq)
        self.i = 0

    def select(self, kind, own, mu, a, allowed, values="corr"):
        t = int(self.seq[self.i])
        self.i += 1
        return t


class Result(dict):
    """s (dense N), S (sorted support), iters, trace [(kind, margin)], near_ties, min_margin,
    resid (final ||y - A s||)."""


def _finish(op, y, S, sS, iters, trace):
    s = np.zeros(op.N)
    s[S] = sS
    margins = [m for _, m in trace]
    return Result(s=s, S=np.asarray(S, dtype=np.int64), iters=iters, trace=trace,
                  near_ties=int(sum(m <= NEAR_TIE for m in margins)),
                  min_margin=float(min(margins)) if margins else 1.0,
                  resid=float(np.linalg.norm(y - op.apply(s))))


def _warm(S_new, S_old, s_old):
    """Start for CG on S_new: the old solution where S_new keeps an old index, 0 elsewhere."""
    x0 = np.zeros(len(S_new))
    if len(S_old):
        pos = np.searchsorted(S_old, S_new)
        pos = np.minimum(pos, len(S_old) - 1)
        hit = S_old[pos] == S_new
        x0[hit] = s_old[pos[hit]]
    return x0


def omp(op, y, K, ls_method="auto", replay=None, on_step=None, policy=None):
    """OMP (Sec. II, Algorithm 1 outer loop).  `replay[i]` forces the i-th selected index
    (shorthand for policy=ForcedSequence(replay)).  `on_step(i, S, sS, r)` is called after each
    iteration (used by invariant tests).  ls_method "auto" solves every LS(S) by QR of A_S
    when M K <= 2.5e5 and otherwise by the growing Cholesky factor (a QR per step would cost
    O(M K^3) over the run); "grow" forces the latter."""
    y = np.asarray(y, dtype=np.float64)
    if policy is None:
        policy = ForcedSequence(replay) if replay is not None else OwnChoice()
    grow = ls_method == "grow" or (ls_method == "auto" and op.M * K > 250_000)
    chol = _ls.GrowingCholesky(op, y, capacity=max(K, 1)) if grow else None
    r = y.copy()
    S = np.zeros(0, dtype=np.int64)
    sS = np.zeros(0)
    trace = []
    for i in range(K):
        a = np.abs(op.apply_t(r))
        allowed = np.ones(op.N, dtype=bool)
        allowed[S] = False
        t, mu = _argmax_lowest(a, allowed)
        t = int(policy.select("argmax", t, mu, a, allowed, "corr"))
        trace.append(("argmax", mu))
        if grow:
            chol.add(t)
            S, sS = chol.solve()
        else:
            S = np.sort(np.append(S, t))
            sS = _ls.ls(op, S, y, ls_method)
        r = y - op.apply_support(S, sS)
        if on_step is not None:
            on_step(i, S, sS, r)
    return _finish(op, y, S, sS, K, trace)


def _topk(policy, a, allowed, K, trace, values):
    pick, mu = topk_lowest(a, allowed, K)
    trace.append(("topk", mu))
    return np.sort(np.asarray(policy.select("topk", pick, mu, a, allowed, values), dtype=np.int64))


def sp(op, y, K, ls_method="auto", L_max=50, policy=None):
    """Subspace Pursuit with the stopping rule stated in the module docstring."""
    y = np.asarray(y, dtype=np.float64)
    policy = policy or OwnChoice()
    trace = []
    everything = np.ones(op.N, dtype=bool)
    S = _topk(policy, np.abs(op.apply_t(y)), everything, K, trace, "corr")
    sS = _ls.ls(op, S, y, ls_method)
    r = y - op.apply_support(S, sS)
    rn = float(np.linalg.norm(r))
    it = 0
    while it < L_max:
        it += 1
        allowed = np.ones(op.N, dtype=bool)
        allowed[S] = False
        T = _topk(policy, np.abs(op.apply_t(r)), allowed, K, trace, "corr")
        St = np.union1d(S, T)
        u = _ls.ls(op, St, y, ls_method, x0=_warm(St, S, sS))
        ua = np.zeros(op.N)
        ua[St] = np.abs(u)
        inside = np.zeros(op.N, dtype=bool)
        inside[St] = True
        Sp = _topk(policy, ua, inside, K, trace, "coef")
        sp_ = _ls.ls(op, Sp, y, ls_method, x0=_warm(Sp, St, u))
        rp = y - op.apply_support(Sp, sp_)
        rpn = float(np.linalg.norm(rp))
        same = np.array_equal(Sp, S)
        mu = 1.0 if same else _test_margin(rn, rpn)
        stop = bool(policy.decide("stop", same or rpn >= rn, mu, None if same else (rn, rpn)))
        trace.append(("stop", mu))
        if stop:
            break
        S, sS, r, rn = Sp, sp_, rp, rpn
    return _finish(op, y, S, sS, it, trace)


def ompr(op, y, K, ls_method="auto", T_max=100, l=1, policy=None):
    """OMP with Replacement (eta = 1) as stated in the module docstring: one swap per iteration
    for l = 1; for l > 1 the OMPR(l) step of Jain, Tewari & Dhillon (2011): J = the l largest
    |z| outside S, S' = the K largest |z| over S u J, stop when S' = S."""
    y = np.asarray(y, dtype=np.float64)
    policy = policy or OwnChoice()
    trace = []
    S = _topk(policy, np.abs(op.apply_t(y)), np.ones(op.N, dtype=bool), K, trace, "corr")
    sS = _ls.ls(op, S, y, ls_method)
    r = y - op.apply_support(S, sS)
    it = 0
    if l > 1:
        while it < T_max:
            z = op.apply_t(r)
            z[S] += sS
            a = np.abs(z)
            inside = np.zeros(op.N, dtype=bool)
            inside[S] = True
            J = _topk(policy, a, ~inside, min(l, op.N - K), trace, "corr")
            union = inside.copy()
            union[J] = True
            S_new = _topk(policy, a, union, K, trace, "coef")
            same = np.array_equal(S_new, S)
            stop = bool(policy.decide("stop", same, 1.0, None))
            trace.append(("stop", 1.0))
            if stop:
                break
            it += 1
            sS = _ls.ls(op, S_new, y, ls_method, x0=_warm(S_new, S, sS))
            S = S_new
            r = y - op.apply_support(S, sS)
        return _finish(op, y, S, sS, it, trace)
    while it < T_max:
        z = op.apply_t(r)
        z[S] += sS
        a = np.abs(z)
        inside = np.zeros(op.N, dtype=bool)
        inside[S] = True
        j, mu_j = _argmax_lowest(a, ~inside)
        j = int(policy.select("argmax", j, mu_j, a, ~inside, "corr"))
        i, mu_i = _argmin_lowest(a, inside)
        i = int(policy.select("argmin", i, mu_i, a, inside, "coef"))
        mu_swap = _test_margin(a[i], a[j])
        trace.append(("argmax", mu_j))
        trace.append(("argmin", mu_i))
        trace.append(("swap", mu_swap))
        if not policy.decide("swap", bool(a[j] > a[i]), mu_swap, (float(a[i]), float(a[j]), len(S))):
            break
        it += 1
        S_new = np.sort(np.append(S[S != i], j))
        sS = _ls.ls(op, S_new, y, ls_method, x0=_warm(S_new, S, sS))
        S = S_new
        r = y - op.apply_support(S, sS)
    return _finish(op, y, S, sS, it, trace)


def cosamp(op, y, K, ls_method="auto", L_max=50, policy=None):
    """CoSaMP with the reading stated in the module docstring."""
    y = np.asarray(y, dtype=np.float64)
    policy = policy or OwnChoice()
    trace = []
    everything = np.ones(op.N, dtype=bool)
    S = np.zeros(0, dtype=np.int64)
    sS = np.zeros(0)
    r = y.copy()
    rn = float(np.linalg.norm(r))
    it = 0
    while it < L_max:
        it += 1
        Om = _topk(policy, np.abs(op.apply_t(r)), everything, 2 * K, trace, "corr")
        T = np.union1d(S, Om)
        b = _ls.ls(op, T, y, ls_method, x0=_warm(T, S, sS))
        ba = np.zeros(op.N)
        ba[T] = np.abs(b)
        inside = np.zeros(op.N, dtype=bool)
        inside[T] = True
        Sp = _topk(policy, ba, inside, K, trace, "coef")
        sp_ = b[np.searchsorted(T, Sp)]
        rp = y - op.apply_support(Sp, sp_)
        rpn = float(np.linalg.norm(rp))
        same = np.array_equal(Sp, S)
        mu = 1.0 if same else _test_margin(rn, rpn)
        stop = bool(policy.decide("stop", same or rpn >= rn, mu, None if same else (rn, rpn)))
        trace.append(("stop", mu))
        if stop:
            break
        S, sS, r, rn = Sp, sp_, rp, rpn
    return _finish(op, y, S, sS, it, trace)


def recover(op, y, K, algo, **kw):
    return {"omp": omp, "sp": sp, "ompr": ompr, "cosamp": cosamp}[algo](op, y, K, **kw)
