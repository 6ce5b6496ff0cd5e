"""CPU-side checks of the C-ABI library: it loads, exports every declared entry point, and its
host-side random draws equal the oracle's independent implementation bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import rng
from paper_1509_03979_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(cs_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1509_03979_gb300 import build
    build.build()
    return binding.lib()


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in binding.SIGNATURES, n


@pytest.mark.parametrize("N,M,seed", [(16, 8, 1), (4096, 1024, 0x0C5001), (1 << 14, 1 << 12, 99),
                                      (1 << 18, 1 << 16, 0x0C5002), (1000, 300, 5), (999, 333, 6), (4095, 17, 7)])
def test_operator_draws_match_oracle(lib, N, M, seed):
    om, d = binding.operator_draws(N, M, seed)
    assert np.array_equal(om.astype(np.int64), rng.omega(N, M, seed))
    assert np.array_equal(d.astype(np.float64), rng.signs(N, seed))


@pytest.mark.parametrize("N,M,code", [(4097, 8, 2), (8, 4, 2), (1 << 25, 8, 2), (3 << 20, 8, 2), (64, 0, 1),
                                      (64, 65, 1), (1000, 1001, 1)])
def test_invalid_sizes_rejected_without_gpu(lib, N, M, code):
    om = np.zeros(max(M, 1), dtype=np.int32)
    st = lib.cs_operator_draws(N, M, 1, om.ctypes.data_as(ctypes.c_void_p), None)
    assert st == code
    assert len(lib.cs_last_error()) > 0


@pytest.mark.parametrize("N,seed", [(16, 1), (4096, 0x0C5001), (1 << 16, 77)])
def test_permutation_draw_matches_oracle(lib, N, seed):
    p = np.zeros(N, dtype=np.int32)
    assert lib.cs_operator_perm(N, seed, p.ctypes.data_as(ctypes.c_void_p)) == 0
    assert np.array_equal(p.astype(np.int64), rng.perm(N, seed))


def test_launch_counter_starts_at_zero_without_a_gpu(lib):
    # nothing can launch on a machine without a GPU; the counter is process-wide
    assert lib.cs_launch_count() == 0


@pytest.mark.parametrize("Bn,N,K,null_c,code", [(-1, 16, 1, False, 1), (1, 0, 0, False, 1), (1, (1 << 30) + 1, 1, False, 1),
                                                (1, 16, 17, False, 1), (1, 16, -1, False, 1), (2, 16, 4, True, 1),
                                                (0, 16, 4, True, 0), (3, 16, 0, True, 0)])
def test_select_arguments_checked_without_gpu(lib, Bn, N, K, null_c, code):
    # argument errors come back before any device work; B = 0 or K = 0 is a no-op
    c = None if null_c else ctypes.c_void_p(16)
    st = lib.cs_select_topk_batched(Bn, N, K, c, None, None if null_c else ctypes.c_void_p(16), None)
    assert st == code
    if code:
        assert len(lib.cs_last_error()) > 0
