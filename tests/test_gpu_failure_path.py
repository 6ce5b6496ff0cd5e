"""GPU: the bounded device wait (the streamed path's grid barrier poll) ends on its own and
reports CS_ERR_TIMEOUT when nothing sets its flag, without faulting or hanging the GPU; the
context stays usable afterwards."""
import time

import numpy as np
import pytest

from tests.gpu_common import APPLY_TOL, rel, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CS_OK, CS_ERR_TIMEOUT = 0, 5


@pytest.fixture(scope="module")
def B():
    from paper_1509_03979_gb300 import binding
    binding.lib()
    return binding


def test_wait_on_a_flag_nothing_sets_times_out(B):
    lib = B.lib()
    t0 = time.time()
    assert lib.cs_probe_bounded_wait(1 << 16, 0) == CS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    assert b"ran out" in lib.cs_last_error()
    assert lib.cs_probe_bounded_wait(1 << 16, 1) == CS_OK
    assert lib.cs_probe_bounded_wait(0, 1) != CS_OK          # argument check


def test_context_usable_after_a_timeout(B):
    import oracle
    assert B.lib().cs_probe_bounded_wait(1 << 12, 0) == CS_ERR_TIMEOUT
    op = B.Operator(4096, 1024, 3)
    ref = oracle.Operator(4096, 1024, 3)
    x = np.random.default_rng(0).standard_normal(4096).astype(np.float32)
    assert rel(op.apply(to_dev(x)).cpu().numpy(), ref.apply(x.astype(np.float64))) <= APPLY_TOL
    op.sync()
