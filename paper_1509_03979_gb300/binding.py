"""Thin ctypes binding over the C ABI in include/cs_gb300.h (argument marshalling only).

Every computation runs in the CUDA library libcs_gb300.so built from csrc/; this module only
checks tensor shapes, dtypes and devices, passes raw pointers, and attaches the calls to
PyTorch's current CUDA stream.  If the library is missing, every call raises: there is no
CPU fallback.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcs_gb300.so")

OMP, SP, OMPR, COSAMP = 0, 1, 2, 3
ALGOS = {"omp": OMP, "sp": SP, "ompr": OMPR, "cosamp": COSAMP}


class CsStats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("cg_iters_total", ctypes.c_int32),
                ("cg_maxit_hits", ctypes.c_int32), ("near_ties", ctypes.c_int32),
                ("final_resid", ctypes.c_float), ("min_margin", ctypes.c_float),
                ("status", ctypes.c_int32), ("transforms", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_I64, _U64, _I32, _F32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "cs_op_create": (_P, [_I64, _I64, _U64]),
    "cs_op_create_ex": (_P, [_I64, _I64, _U64, _I32]),
    "cs_op_create_basis": (_P, [_I64, _I64, _U64, _I32, _I32]),
    "cs_operator_perm": (_I32, [_I64, _U64, _P]),
    "cs_op_export_perm": (_I32, [_P, _P]),
    "cs_op_destroy": (None, [_P]),
    "cs_op_set_stream": (_I32, [_P, _P]),
    "cs_op_apply": (_I32, [_P, _P, _P]),
    "cs_op_apply_t": (_I32, [_P, _P, _P]),
    "cs_op_export": (_I32, [_P, _P, _P]),
    "cs_op_apply_batched": (_I32, [_P, _I32, _P, _P]),
    "cs_op_apply_t_batched": (_I32, [_P, _I32, _P, _P]),
    "cs_op_concurrency": (_I32, [_P]),
    "cs_op_set_batched_impl": (_I32, [_P, _I32]),
    "cs_op_set_cg_tol_mode": (_I32, [_P, _I32]),
    "cs_op_set_ompr_replacements": (_I32, [_P, _I32]),
    "cs_op_set_cluster_size": (_I32, [_P, _I32]),
    "cs_op_cluster_size": (_I32, [_P]),
    "cs_op_tune_recover": (_I32, [_P, _I32, _I32, _F32, _I32, _P]),
    "cs_op_tune_batched": (_I32, [_P, _I32, _P]),
    "cs_operator_draws": (_I32, [_I64, _I64, _U64, _P, _P]),
    "cs_recover": (_I32, [_P, _P, _I32, _I32, _F32, _I32, _P, _P]),
    "cs_recover_noalloc": (_I32, [_P, _P, _I32, _I32, _F32, _I32, _P, _P]),
    "cs_op_set_trace": (_I32, [_P, _P, _I64]),
    "cs_op_set_outer_cap": (_I32, [_P, _I32]),
    "cs_recover_batched": (_I32, [_I32, _P, _P, _P, _P, _F32, _I32, _P, _P, _P]),
    "cs_ls_solve": (_I32, [_P, _P, _I32, _P, _F32, _I32, _P]),
    "cs_ls_backward": (_I32, [_P, _P, _I32, _P, _F32, _I32, _P]),
    "cs_ls_solve_batched": (_I32, [_P, _I32, _P, _I32, _P, _F32, _I32, _P]),
    "cs_ls_backward_batched": (_I32, [_P, _I32, _P, _I32, _P, _F32, _I32, _P]),
    "cs_get_stats": (_I32, [_P, _P]),
    "cs_op_sync": (_I32, [_P]),
    "cs_select_topk_batched": (_I32, [_I32, _I64, _I32, _P, _P, _P, _P]),
    "cs_probe_bounded_wait": (_I32, [_U64, _I32]),
    "cs_last_error": (ctypes.c_char_p, []),
    "cs_launch_count": (ctypes.c_int64, []),
}


def lib():
    """Load libcs_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(status):
    if status != 0:
        raise RuntimeError(f"cs_gb300 error {status}: {lib().cs_last_error().decode()}")


def _dev(t, dtype, n=None, name="tensor"):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def launch_count():
    """Kernel launches this library has issued in this process (cs_launch_count)."""
    return int(lib().cs_launch_count())


def operator_draws(N, M, seed):
    """The operator's Omega (sorted int32 [M]) and d (+-1 int8 [N]), computed on the host."""
    import numpy as np
    om = np.zeros(M, dtype=np.int32)
    d = np.zeros(N, dtype=np.int8)
    _check(lib().cs_operator_draws(N, M, seed, om.ctypes.data_as(_P), d.ctypes.data_as(_P)))
    return om, d


class Operator:
    """A = P_Omega C_N diag(d) on the current CUDA device (Sec. III-A, Eq. 7)."""

    RANDOMIZERS = {"signs": 0, "perm": 1}
    BASES = {None: 0, "dct": 1, "dct2d": 2}

    def __init__(self, N, M, seed, randomizer="signs", psi=None):
        """randomizer: 'signs' (R = diag(d), the default) or 'perm' (R a random permutation);
        psi: None (s sparse itself), 'dct' (s the DCT coefficients of x = C_N^T s) or
        ('dct2d', n1, n2) (s the 2-D DCT coefficients of an n1 x n2 row-major image)."""
        self.N, self.M, self.seed = int(N), int(M), int(seed)
        self.randomizer = randomizer
        self.psi = psi
        if psi is not None:
            if randomizer != "signs":
                raise ValueError("a sparsifying basis takes the sign randomiser")
            kind, n1 = (psi, 0) if psi == "dct" else (psi[0], int(psi[1]))
            if kind == "dct2d" and n1 * int(psi[2]) != self.N:
                raise ValueError("psi=('dct2d', n1, n2) needs n1 n2 = N")
            h = lib().cs_op_create_basis(self.N, self.M, self.seed, self.BASES[kind], n1)
        else:
            h = lib().cs_op_create_ex(self.N, self.M, self.seed, self.RANDOMIZERS[randomizer])
        if not h:
            raise RuntimeError(f"cs_op_create failed: {lib().cs_last_error().decode()}")
        self._h = ctypes.c_void_p(h)

    def export_perm(self):
        import numpy as np
        p = np.zeros(self.N, dtype=np.int32)
        _check(lib().cs_op_export_perm(self._h, p.ctypes.data_as(ctypes.c_void_p)))
        return p

    def close(self):
        if getattr(self, "_h", None):
            lib().cs_op_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def _stream(self):
        _check(lib().cs_op_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def apply(self, x, out=None):
        out = torch.empty(self.M, dtype=torch.float32, device=x.device) if out is None else out
        self._stream()
        _check(lib().cs_op_apply(self._h, _dev(x, torch.float32, self.N, "x"), _dev(out, torch.float32, self.M, "y")))
        return out

    def apply_t(self, u, out=None):
        out = torch.empty(self.N, dtype=torch.float32, device=u.device) if out is None else out
        self._stream()
        _check(lib().cs_op_apply_t(self._h, _dev(u, torch.float32, self.M, "u"), _dev(out, torch.float32, self.N, "x")))
        return out

    def apply_batched(self, X, out=None):
        """Y[b] = A X[b] for X of shape [B, N]."""
        Bn = X.shape[0]
        out = torch.empty((Bn, self.M), dtype=torch.float32, device=X.device) if out is None else out
        self._stream()
        _check(lib().cs_op_apply_batched(self._h, Bn, _dev(X, torch.float32, Bn * self.N, "X"),
                                         _dev(out, torch.float32, Bn * self.M, "Y")))
        return out

    def apply_t_batched(self, U, out=None):
        """X[b] = A^T U[b] for U of shape [B, M]."""
        Bn = U.shape[0]
        out = torch.empty((Bn, self.N), dtype=torch.float32, device=U.device) if out is None else out
        self._stream()
        _check(lib().cs_op_apply_t_batched(self._h, Bn, _dev(U, torch.float32, Bn * self.M, "U"),
                                           _dev(out, torch.float32, Bn * self.N, "X")))
        return out

    def concurrency(self):
        """Signals of this size the GPU runs at once (resident clusters)."""
        return int(lib().cs_op_concurrency(self._h))

    def set_trace(self, trace):
        """Record the selection trace of later recoveries into `trace` (a CUDA int32 tensor;
        None disables it).  The tensor must outlive the recoveries that write it."""
        if trace is None:
            _check(lib().cs_op_set_trace(self._h, None, 0))
            self._trace = None
            return
        _check(lib().cs_op_set_trace(self._h, _dev(trace, torch.int32, None, "trace"), int(trace.numel())))
        self._trace = trace

    def set_outer_cap(self, cap):
        """Cap on SP / CoSaMP rounds and OMPR swaps of later recoveries (0: 50 and 100)."""
        _check(lib().cs_op_set_outer_cap(self._h, int(cap)))

    def set_ompr_replacements(self, l):
        """Replacements per OMPR round (1: single swap; l > 1: OMPR(l))."""
        _check(lib().cs_op_set_ompr_replacements(self._h, int(l)))

    def set_cg_tol_mode(self, mode):
        """CG stopping rule of later recover / LS calls: 'relative' (to ||b||) or 'absolute'."""
        _check(lib().cs_op_set_cg_tol_mode(self._h, {"relative": 0, "absolute": 1}[mode]))

    def set_cluster_size(self, P):
        """CTAs per signal of the cluster engine (0: the smallest that holds the transform)."""
        _check(lib().cs_op_set_cluster_size(self._h, int(P)))

    def cluster_size(self):
        return int(lib().cs_op_cluster_size(self._h))

    def tune_recover(self, K, algo="omp", cg_tol=1e-6, cg_maxit=100):
        """Time a recovery for every valid cluster size, keep the fastest; returns {P: ms}."""
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        ms = (ctypes.c_float * 5)()
        self._stream()
        _check(lib().cs_op_tune_recover(self._h, int(K), a, float(cg_tol), int(cg_maxit), ms))
        return {1 << i: ms[i] for i in range(5) if ms[i] >= 0}

    BATCHED_IMPLS = {"auto": 0, "cluster": 1, "streamed": 2}

    def set_batched_impl(self, impl):
        """Implementation of apply_batched / apply_t_batched: 'auto', 'cluster' or 'streamed'."""
        _check(lib().cs_op_set_batched_impl(self._h, self.BATCHED_IMPLS[impl]))

    TUNE_CANDIDATES = ("cluster", "streamed x1", "streamed x2", "streamed x4", "streamed x8")

    def tune_batched(self, B):
        """Time every batched candidate on B vectors and keep the fastest (per direction).
        Returns {"A": {candidate: ms}, "AT": {...}} for the candidates that apply."""
        ms = (ctypes.c_float * 10)()
        self._stream()
        _check(lib().cs_op_tune_batched(self._h, int(B), ms))
        out = {}
        for d, name in enumerate(("A", "AT")):
            out[name] = {c: ms[5 * d + i] for i, c in enumerate(self.TUNE_CANDIDATES) if ms[5 * d + i] >= 0}
        return out

    def export(self):
        import numpy as np
        om = np.zeros(self.M, dtype=np.int32)
        d = np.zeros(self.N, dtype=np.int8)
        _check(lib().cs_op_export(self._h, om.ctypes.data_as(_P), d.ctypes.data_as(_P)))
        return om, d

    def recover(self, y, K, algo="omp", cg_tol=1e-6, cg_maxit=100, s_out=None, support_out=None):
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        s_out = torch.empty(self.N, dtype=torch.float32, device=y.device) if s_out is None else s_out
        support_out = (torch.empty(max(K, 1), dtype=torch.int32, device=y.device)
                       if support_out is None else support_out)
        self._stream()
        _check(lib().cs_recover(self._h, _dev(y, torch.float32, self.M, "y"), int(K), a, float(cg_tol),
                                int(cg_maxit), _dev(s_out, torch.float32, self.N, "s_out"),
                                _dev(support_out, torch.int32, None, "support_out")))
        return s_out, support_out[:K]

    def recover_noalloc(self, y, K, algo="omp", cg_tol=1e-6, cg_maxit=100, s_out=None, support_out=None):
        """cs_recover_noalloc: the same recovery with scratch from the library's fixed device
        array (no device allocation by the call; N <= 65536).  Outputs must be preallocated by
        a caller that cannot allocate; they are allocated here only when not given."""
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        s_out = torch.empty(self.N, dtype=torch.float32, device=y.device) if s_out is None else s_out
        support_out = (torch.empty(max(K, 1), dtype=torch.int32, device=y.device)
                       if support_out is None else support_out)
        self._stream()
        _check(lib().cs_recover_noalloc(self._h, _dev(y, torch.float32, self.M, "y"), int(K), a, float(cg_tol),
                                        int(cg_maxit), _dev(s_out, torch.float32, self.N, "s_out"),
                                        _dev(support_out, torch.int32, None, "support_out")))
        return s_out, support_out[:K]

    def ls_solve(self, support, y, cg_tol=1e-6, cg_maxit=100, out=None):
        """Batched when y is [B, M] and support is [B, k]."""
        batched = y.dim() == 2
        B = y.shape[0] if batched else 1
        k = support.shape[-1]
        out = torch.empty((B, k) if batched else (k,), dtype=torch.float32, device=y.device) if out is None else out
        self._stream()
        _check(lib().cs_ls_solve_batched(self._h, B, _dev(support, torch.int32, B * k, "support"), k,
                                         _dev(y, torch.float32, B * self.M, "y"), float(cg_tol), int(cg_maxit),
                                         _dev(out, torch.float32, B * k, "out")))
        return out

    def ls_backward(self, support, g, cg_tol=1e-6, cg_maxit=100, out=None):
        batched = g.dim() == 2
        B = g.shape[0] if batched else 1
        k = support.shape[-1]
        out = (torch.empty((B, self.M) if batched else (self.M,), dtype=torch.float32, device=g.device)
               if out is None else out)
        self._stream()
        _check(lib().cs_ls_backward_batched(self._h, B, _dev(support, torch.int32, B * k, "support"), k,
                                            _dev(g, torch.float32, B * k, "g"), float(cg_tol), int(cg_maxit),
                                            _dev(out, torch.float32, B * self.M, "dy")))
        return out

    def stats(self):
        st = CsStats()
        _check(lib().cs_get_stats(self._h, ctypes.byref(st)))
        return st.as_dict()

    def sync(self):
        """Wait for this operator's stream; raises if its last launch failed or timed out."""
        _check(lib().cs_op_sync(self._h))


def select_topk_batched(c, K, exclude=None, out=None):
    """cs_select_topk_batched: for every row of c ([B, N] float32, CUDA) the K indices with the
    largest |c| outside `exclude` (int32 [B, ceil(N/32)] bit words, or None), ties to the lowest
    index, ascending; -1 past a row's eligible count.  Returns int32 [B, K] on the current stream."""
    if c.dim() != 2:
        raise ValueError("c must be [B, N]")
    B, N = c.shape
    _dev(c, torch.float32, name="c")
    W = (N + 31) // 32
    ex = ctypes.c_void_p(0)
    if exclude is not None:
        ex = _dev(exclude, torch.int32, B * W, name="exclude")
    out = out if out is not None else torch.empty((B, K), dtype=torch.int32, device=c.device)
    _dev(out, torch.int32, B * K, name="out")
    stream = ctypes.c_void_p(torch.cuda.current_stream(c.device).cuda_stream)
    _check(lib().cs_select_topk_batched(B, N, K, ctypes.c_void_p(c.data_ptr()), ex,
                                        ctypes.c_void_p(out.data_ptr()), stream))
    return out


def recover_batched(ops, ys, Ks, algos, cg_tol=1e-6, cg_maxit=100, s_outs=None, supports=None, want_stats=False):
    """Recover B independent signals (each with its own operator) in one persistent launch
    per cluster size.  Returns (s_outs, supports[, stats])."""
    B = len(ops)
    s_outs = s_outs or [torch.empty(op.N, dtype=torch.float32, device=y.device) for op, y in zip(ops, ys)]
    supports = supports or [torch.empty(max(k, 1), dtype=torch.int32, device=y.device) for k, y in zip(Ks, ys)]
    for op in ops:
        op._stream()
    arr = lambda ctype, vals: (ctype * B)(*vals)
    h = arr(_P, [op.handle.value for op in ops])
    yp = arr(_P, [_dev(y, torch.float32, op.M, "y").value for op, y in zip(ops, ys)])
    sp = arr(_P, [_dev(s, torch.float32, op.N, "s_out").value for op, s in zip(ops, s_outs)])
    kp = arr(_P, [_dev(t, torch.int32, None, "support").value for t in supports])
    Karr = arr(_I32, [int(k) for k in Ks])
    Aarr = arr(_I32, [ALGOS[a] if isinstance(a, str) else int(a) for a in algos])
    st = (CsStats * B)() if want_stats else None
    _check(lib().cs_recover_batched(B, h, yp, Karr, Aarr, float(cg_tol), int(cg_maxit), sp, kp,
                                    st if want_stats else None))
    out = (s_outs, [t[:k] for t, k in zip(supports, Ks)])
    if want_stats:
        return out + ([s.as_dict() for s in st],)
    return out


class CGLeastSquares(torch.autograd.Function):
    """s_S = LS(y; S) on a fixed support through the CUDA CG solver; backward applies the
    hand-written adjoint dy = A_S (A_S^T A_S)^{-1} g (the support gets no gradient)."""

    @staticmethod
    def forward(ctx, y, support, op, cg_tol=1e-6, cg_maxit=100):
        ctx.op, ctx.cg_tol, ctx.cg_maxit = op, cg_tol, cg_maxit
        ctx.save_for_backward(support)
        return op.ls_solve(support, y.contiguous(), cg_tol, cg_maxit)

    @staticmethod
    def backward(ctx, g):
        (support,) = ctx.saved_tensors
        dy = ctx.op.ls_backward(support, g.contiguous(), ctx.cg_tol, ctx.cg_maxit)
        return dy, None, None, None, None
