"""The device-side failure path, tested without a GPU fault: a bounded wait
that nothing completes gives up (about a second), the next sync reports
TSK_ERR_TIMEOUT through the C ABI, the error word is cleared, and the context
keeps working."""
import ctypes as C

import numpy as np
import pytest

from helpers import check_profile

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03393_gb300 import build
    build.build()
    import paper_2311_03393_gb300 as t
    return t


def test_a_bounded_wait_that_runs_out_is_reported_and_the_context_survives(tsk):
    from paper_2311_03393_gb300 import _native as N
    lib = N.lib()
    h = tsk.context()
    assert lib.tsk_selftest_timeout(h) == N.TSK_OK
    assert lib.tsk_sync(h, C.c_double(30.0)) == 5  # TSK_ERR_TIMEOUT
    assert b"wait" in lib.tsk_last_error(h)
    assert lib.tsk_sync(h, C.c_double(30.0)) == N.TSK_OK  # the error word was cleared
    # the same context still computes correct profiles
    rng = np.random.default_rng(71)
    x = np.cumsum(rng.normal(size=3000)).astype(np.float32)
    P, I = tsk.mp_selfjoin(torch.from_numpy(x).cuda(), [3000], 50, 12)
    tsk.sync()
    l = 3000 - 50 + 1
    check_profile(x.astype(np.float64), 50, 12, P.cpu().numpy()[:l], I.cpu().numpy()[:l], rows=np.arange(0, l, 5))
