"""Selection-by-selection parity of a GPU recovery with the FP64 oracle (test infrastructure
only: used by the tests, the smoke check and the benchmark's parity and CPU-baseline legs).

The GPU decoders write a selection trace (cs_op_set_trace): every argmax, argmin, top-K and
stop / swap test in decoder order, with its FP32 margin.  `GpuReplay` is an oracle selection
policy that walks that trace while the oracle runs the same decoder:

  * where the oracle's margin exceeds NEAR_TIE (1e-3) the GPU must have made the oracle's
    choice exactly (the same index, the same set, the same stop decision);
  * at a near-tie any member of the tied set is valid: the GPU's choice is checked to lie
    within the tie band (|a_e - a_ref| <= NEAR_TIE a_ref for every index where the two
    choices differ) and the oracle continues with the GPU's choice (replay), so that the rest
    of the run, and the final s_hat, stay comparable.

`check_recovery` runs the replayed oracle and asserts the final support equals the GPU's and
s_hat is within the given relative L2 tolerance, and that the GPU's margins agree with the
oracle's.
"""
import numpy as np

from . import greedy

NEAR_TIE = greedy.NEAR_TIE
KINDS = {1: "argmax", 2: "argmin", 3: "topk", 4: "stop", 5: "swap"}
HEADER = 4


def trace_words(N, K, algo, L_max=50, T_max=100, ompr_l=1):
    """A capacity that holds every record the decoder can write."""
    W = (N + 31) // 32
    if algo == "omp":
        return HEADER + 4 * K + 16
    if algo == "ompr" and ompr_l <= 1:
        return HEADER + (4 + W) + 12 * T_max + 16
    rounds = T_max if algo == "ompr" else L_max
    return HEADER + (2 * rounds + 2) * (4 + W) + 4 * rounds + 16


def parse_trace(tr):
    """Records of a trace (int32 numpy array) as dicts {kind, mu, aux, idx (top-K: indices)}."""
    tr = np.asarray(tr).astype(np.int64) & 0xFFFFFFFF
    used, nrec, over, W = (int(v) for v in tr[:HEADER])
    assert not over, "the selection trace overflowed its buffer"
    recs, off = [], HEADER
    for _ in range(nrec):
        kind, pay, mu_bits, aux = (int(v) for v in tr[off:off + 4])
        mu = float(np.array([mu_bits], dtype=np.uint32).view(np.float32)[0])
        r = {"kind": KINDS[kind], "mu": mu, "aux": aux}
        if kind == 3:
            words = tr[off + 4:off + 4 + pay].astype(np.uint32)
            bits = np.unpackbits(words.view(np.uint8), bitorder="little")
            r["idx"] = np.flatnonzero(bits).astype(np.int64)
        recs.append(r)
        off += 4 + pay
    assert off == used, (off, used)
    return recs


class Floors:
    """Absolute resolution of the FP32 values the GPU selects on, for a recovery of y with CG
    run to relative tolerance t (floored at 2e-6, about 32 FP32 roundings).  The GPU's
    least-squares coefficients carry the CG error: ||dx|| <= t ||b|| / lambda_min(A_S^T A_S)
    with ||b|| ~ sqrt(M/N) ||y|| and lambda_min ~ (M/N) (1 - sqrt(k/M))^2 >= 0.3 M/N here, so a
    coefficient is resolved to about 3.3 t ||y|| sqrt(N/M) / sqrt(k) and, taking 8 standard
    deviations, coef(k) = 25 t ||y|| sqrt(N/M) / sqrt(k).  A correlation a_j^T r off the support
    sees that error through A: corr = 8 t ||y|| / sqrt(N).  Residual norms: resid = 8 t ||y||.
    Below these, orderings are set by rounding, not by the data."""

    def __init__(self, y, N, M, cg_tol):
        t = max(float(cg_tol), 2e-6)
        ny = float(np.linalg.norm(y))
        self.corr = 8.0 * t * ny / np.sqrt(N)
        self._coef = 25.0 * t * ny * np.sqrt(N / M)
        self.resid = 8.0 * t * ny

    def coef(self, k):
        return self._coef / np.sqrt(max(int(k), 1))

    def of(self, values, k):
        return self.corr if values == "corr" else self.coef(k)


class GpuReplay(greedy.OwnChoice):
    """Oracle policy that checks every GPU choice and continues with it (see module text).

    A selection counts as a near-tie when its relative margin is <= NEAR_TIE or, with `floors`,
    when the gap that decides it is within twice the FP32 resolution of the values; there any
    choice inside the tie band (relative NEAR_TIE plus twice the resolution) is valid."""

    def __init__(self, records, floors=None):
        self.recs = records
        self.i = 0
        self.floors = floors
        self.selections = 0
        self.near = 0
        self.floor_ties = 0                 # near-ties by the absolute resolution only
        self.diverged = []                  # (position, kind, oracle margin) where the GPU chose otherwise
        self.mu_pairs = []                  # (oracle margin, GPU margin)

    def _next(self, kinds):
        assert self.i < len(self.recs), f"the GPU trace ended after {self.i} records"
        r = self.recs[self.i]
        assert r["kind"] in kinds, (self.i, r["kind"], kinds)
        self.i += 1
        return r

    def _delta(self, values, allowed):
        if self.floors is None:
            return 0.0
        return self.floors.of(values, int(np.count_nonzero(allowed)))

    @staticmethod
    def _gap(kind, own, a, allowed):
        rest = allowed.copy()
        if kind == "topk":
            own = np.asarray(own, dtype=np.int64)
            rest[own] = False
            inner = float(np.min(a[own]))
            outer = float(np.max(a[rest])) if rest.any() else 0.0
            return inner - outer, inner
        rest[own] = False
        if kind == "argmax":
            other = float(np.max(a[rest])) if rest.any() else 0.0
            return float(a[own]) - other, float(a[own])
        other = float(np.min(a[rest])) if rest.any() else np.inf
        return other - float(a[own]), float(a[own])

    def select(self, kind, own, mu, a, allowed, values="corr"):
        r = self._next((kind,))
        self.selections += 1
        self.mu_pairs.append((mu, r["mu"]))
        delta = self._delta(values, allowed)
        gap, ref = self._gap(kind, own, a, allowed)
        near = mu <= NEAR_TIE or gap <= 2.0 * delta
        self.near += int(near)
        self.floor_ties += int(near and mu > NEAR_TIE)
        band = NEAR_TIE * ref + 2.0 * delta
        if kind in ("argmax", "argmin"):
            got = int(r["aux"])
            assert allowed[got], (self.i, kind, got)
            if got != own:
                assert near, f"selection {self.i} ({kind}): GPU {got}, oracle {own}, margin {mu:.3e} > 1e-3"
                assert abs(a[got] - a[own]) <= band, (self.i, kind, got, own, a[got], a[own], band)
                self.diverged.append((self.i, kind, mu))
            return got
        got = r["idx"]
        own = np.asarray(own, dtype=np.int64)
        assert len(got) == len(own) and np.all(allowed[got]), (self.i, len(got), len(own))
        if not np.array_equal(got, own):
            assert near, (f"selection {self.i} (top-K): {len(np.setxor1d(got, own))} indices differ, "
                          f"margin {mu:.3e} > 1e-3, gap {gap:.3e} > 2 x resolution {delta:.3e}")
            diff = np.setxor1d(got, own)
            bad = diff[np.abs(a[diff] - ref) > band]
            assert len(bad) == 0, (self.i, "top-K outside the tie band", bad[:8], band)
            self.diverged.append((self.i, kind, mu))
        return got

    def decide(self, kind, own, mu, vals=None):
        r = self._next((kind,))
        self.mu_pairs.append((mu, r["mu"]))
        got = bool(r["aux"])
        near = mu <= NEAR_TIE
        if not near and vals is not None and self.floors is not None:
            delta = self.floors.resid if kind == "stop" else self.floors.corr + self.floors.coef(vals[2])
            near = abs(vals[0] - vals[1]) <= 2.0 * delta or max(vals[:2]) <= delta
            self.floor_ties += int(near)
        self.near += int(near)
        if got != bool(own):
            assert near, f"test {self.i} ({kind}): GPU {got}, oracle {own}, margin {mu:.3e} > 1e-3"
            self.diverged.append((self.i, kind, mu))
        return got

    def finish(self):
        assert self.i == len(self.recs), f"the GPU made {len(self.recs) - self.i} more selections than the replay"
        mu = np.array(self.mu_pairs, dtype=np.float64).reshape(-1, 2)
        return {"selections": self.selections, "tests": len(self.mu_pairs) - self.selections,
                "near_ties": self.near, "floor_ties": self.floor_ties, "diverged": self.diverged,
                "max_margin_gap": float(np.max(np.abs(mu[:, 0] - mu[:, 1]))) if len(mu) else 0.0}


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def check_recovery(ref_op, y, K, algo, trace, s_gpu, supp_gpu, shat_tol, stats=None,
                   margin_tol=None, cg_tol=1e-6, **kw):
    """Replay the oracle along the GPU's trace and assert parity; returns the report.
    cg_tol: the GPU's relative CG tolerance (sets the FP32 resolution, see Floors); kw go to the
    oracle decoder (ls_method, l, T_max, L_max)."""
    y = np.asarray(y, dtype=np.float64)
    pol = GpuReplay(parse_trace(trace), Floors(y, ref_op.N, ref_op.M, cg_tol))
    ref = greedy.recover(ref_op, np.asarray(y, dtype=np.float64), K, algo, policy=pol, **kw)
    rep = pol.finish()
    supp_gpu = np.sort(np.asarray(supp_gpu, dtype=np.int64))
    assert np.array_equal(supp_gpu, ref["S"]), "final support differs from the replayed oracle"
    err = rel(s_gpu, ref["s"])
    assert err <= shat_tol, f"s_hat rel err {err:.3e} > {shat_tol}"
    rep["rel_err"] = err
    rep["oracle_iters"] = ref["iters"]
    if margin_tol is not None:
        assert rep["max_margin_gap"] <= margin_tol, rep["max_margin_gap"]
    if stats is not None:
        # the device's near-tie count sees the same choices with FP32 margins
        nt = sum(1 for o, g in pol.mu_pairs if g <= NEAR_TIE)
        assert stats["near_ties"] == nt, (stats["near_ties"], nt)
        gm = min((g for _, g in pol.mu_pairs), default=1.0)
        assert abs(stats["min_margin"] - gm) <= 1e-6 * max(1.0, abs(gm)), (stats["min_margin"], gm)
    return rep, ref


# ------------------------------------------------------------- process-pool workers
def replay_job(job):
    """Full replay of one recovery (for a spawn-started process pool): job holds the operator's
    (N, M, op_seed), y, K, algo, the GPU's trace, s_hat, support and statistics."""
    import oracle
    ref_op = oracle.Operator(job["N"], job["M"], job["op_seed"], randomizer=job.get("randomizer", "signs"))
    rep, _ = check_recovery(ref_op, job["y"], job["K"], job["algo"], job["trace"], job["s"], job["supp"],
                            job["shat_tol"], stats=job.get("stats"), cg_tol=job.get("cg_tol", 1e-6),
                            **job.get("kw", {}))
    rep["index"] = job.get("index")
    return rep


def _state_after(records, t, algo):
    """Support the GPU held before its selection t (OMP: t argmax records in; OMPR: swap t,
    1-based, after the initial top-K and t - 1 swaps)."""
    if algo == "omp":
        return np.sort(np.array([r["aux"] for r in records[:t]], dtype=np.int64))
    S = set(records[0]["idx"].tolist())
    for u in range(t - 1):
        j, i, sw = records[1 + 3 * u: 4 + 3 * u]
        assert sw["aux"] == 1
        S.discard(i["aux"])
        S.add(j["aux"])
    return np.array(sorted(S), dtype=np.int64)


def state_job(job):
    """Check one selection of a long OMP or single-swap OMPR run from the GPU's own state: the
    support before it is rebuilt from the trace, LS(S) is solved in FP64 (QR or CG to 1e-13),
    the oracle makes the selection and GpuReplay compares it with the GPU's record (exact above
    the margin, tie band below).  Independent of every other selection, so a sample of them
    checks a trajectory the oracle could not replay end to end."""
    import oracle
    from oracle import ls as _ls
    op = oracle.Operator(job["N"], job["M"], job["op_seed"])
    y = np.asarray(job["y"], dtype=np.float64)
    recs = parse_trace(job["trace"])
    t, algo = job["t"], job["algo"]
    S = _state_after(recs, t, algo)
    sS = _ls.ls(op, S, y) if len(S) else np.zeros(0)
    r = y - op.apply_support(S, sS) if len(S) else y.copy()
    c = op.apply_t(r)
    inside = np.zeros(op.N, dtype=bool)
    inside[S] = True
    floors = Floors(y, op.N, op.M, job.get("cg_tol", 1e-6))
    if algo == "omp":
        pol = GpuReplay([recs[t]], floors)
        t_own, mu = greedy._argmax_lowest(np.abs(c), ~inside)
        pol.select("argmax", t_own, mu, np.abs(c), ~inside, "corr")
    else:
        z = c.copy()
        z[S] += sS
        a = np.abs(z)
        pol = GpuReplay(recs[1 + 3 * (t - 1): 4 + 3 * (t - 1)], floors)
        j, mu_j = greedy._argmax_lowest(a, ~inside)
        j = pol.select("argmax", j, mu_j, a, ~inside, "corr")
        i, mu_i = greedy._argmin_lowest(a, inside)
        i = pol.select("argmin", i, mu_i, a, inside, "coef")
        pol.decide("swap", bool(a[j] > a[i]), greedy._test_margin(a[i], a[j]), (float(a[i]), float(a[j]), len(S)))
    rep = pol.finish()
    rep["t"] = t
    rep["index"] = job.get("index")
    return rep


def run_pool(fn, jobs, workers=None):
    """Map fn over jobs in a process pool started with 'spawn' (the parent holds a CUDA
    context) and single-threaded numpy in each worker."""
    import multiprocessing as mp
    import os
    if not jobs:
        return []
    workers = workers or max(1, min(len(jobs), (os.cpu_count() or 2) - 1))
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            return pool.map(fn, jobs, chunksize=1)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def final_ls_job(job):
    """s_hat of a recovery against the FP64 least-squares solution on the GPU's own support."""
    import oracle
    from oracle import ls as _ls
    op = oracle.Operator(job["N"], job["M"], job["op_seed"])
    S = np.sort(np.asarray(job["supp"], dtype=np.int64))
    assert len(S) == job["K"] and np.all(np.diff(S) > 0)
    full = np.zeros(job["N"])
    full[S] = _ls.ls(op, S, np.asarray(job["y"], dtype=np.float64))
    err = rel(job["s"], full)
    assert err <= job["shat_tol"], (job.get("index"), err)
    return {"index": job.get("index"), "rel_err": err}


def pinv_grad_job(job):
    """FP64 gradient of L(y) = ||LS_S(y) - s_true_S||^2 by the dense QR pseudo-inverse, and, for
    each direction v in job["V"] (rows), the central difference (L(y + eps v) - L(y - eps v)) /
    (2 eps) of the same FP64 L at job["eps"] (exact up to rounding: L is quadratic in y)."""
    import scipy.linalg as sla

    import oracle
    from oracle import adjoint
    op = oracle.Operator(job["N"], job["M"], job["op_seed"])
    S = np.asarray(job["S"], dtype=np.int64)
    y = np.asarray(job["y"], dtype=np.float64)
    t = np.asarray(job["s_true_S"], dtype=np.float64)
    _, g = adjoint.loss_grad_y(op, S, y, t)
    Q, R = np.linalg.qr(op.columns(S), mode="reduced")

    def L(yv):
        d = sla.solve_triangular(R, Q.T @ yv, lower=False) - t
        return float(d @ d)
    eps = float(job.get("eps", 1e-3))
    fd = [(L(y + eps * v) - L(y - eps * v)) / (2.0 * eps) for v in np.asarray(job.get("V", np.zeros((0, len(y)))))]
    return g, np.array(fd)
