"""The allocation-free matrix-profile entry point (mp_selfjoin_static).

Some callers cannot allocate device memory: a monitor that must not allocate
after start-up, code whose device memory belongs to another framework's pool,
or code called back from inside an allocator.  mp_selfjoin_static serves them
from a fixed array in the library's device memory.  Here it is called through
the C ABI on two inputs in a row.  Each result must agree with mp_selfjoin's
and with the float64 oracle's rows (Def. 6) within the parity bar; the second
call also checks that the shared array's leftovers from the first call do not
leak into its result.  This file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from helpers import MP_REL_TOL, check_profile, d_floor

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03393_gb300 import build
    build.build()
    import paper_2311_03393_gb300 as tsk
    from paper_2311_03393_gb300 import _native
    return tsk, _native.lib()


def _static_call(lib, X, n, m, excl):
    P = torch.full((n,), -7.0, device="cuda")
    I = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = lib.mp_selfjoin_static(C.c_void_p(X.data_ptr()), n, m, excl, C.c_void_p(P.data_ptr()),
                                C.c_void_p(I.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    return P, I


def test_static_entry_point_matches_mp_selfjoin_on_two_calls(libs):
    tsk, lib = libs
    m, excl = 100, 25
    floor = d_floor(m)
    for seed, n in ((300, 5000), (301, 2300), (303, 4000)):
        rng = np.random.default_rng(seed)
        if seed == 303:  # a sine with noise 1e-4: near-exact repeats below float32 resolution
            x = (np.sin(2 * np.pi * np.arange(n) / 64) + 1e-4 * rng.normal(size=n)).astype(np.float32)
        else:
            x = np.cumsum(rng.normal(size=n)).astype(np.float32)
        X = torch.from_numpy(x).cuda()
        P, I = _static_call(lib, X, n, m, excl)
        P_ref, I_ref = tsk.mp_selfjoin(X, [n], m, excl)
        torch.cuda.synchronize()
        l = n - m + 1
        P, I = P.cpu().numpy(), I.cpu().numpy()
        P_ref = P_ref.cpu().numpy()
        assert np.all(np.isnan(P[l:])) and np.all(I[l:] == -1)
        # against the existing entry point
        err = np.abs(P[:l] - P_ref[:l]) / np.maximum(P_ref[:l], floor)
        assert err.max() <= MP_REL_TOL, float(err.max())
        # against the oracle, indices included (equal or an equally near neighbour)
        check_profile(x.astype(np.float64), m, excl, P[:l], I[:l], rows=np.arange(0, l, 2))


def test_static_entry_point_after_a_smaller_window_on_the_context_path(libs):
    """The context path's shared-memory limits must not shrink what the static path needs."""
    tsk, lib = libs
    n = 6000
    x = np.cumsum(np.random.default_rng(302).normal(size=n)).astype(np.float32)
    X = torch.from_numpy(x).cuda()
    tsk.mp_selfjoin(X, [n], 16, 4)  # small m first
    m, excl = 1500, 375
    P, I = _static_call(lib, X, n, m, excl)
    torch.cuda.synchronize()
    l = n - m + 1
    check_profile(x.astype(np.float64), m, excl, P.cpu().numpy()[:l], I.cpu().numpy()[:l],
                  rows=np.arange(0, l, 15))


def test_static_entry_point_rejects_inputs_beyond_its_limit(libs):
    _, lib = libs
    n = 65536 + 100  # l = 65537 windows > 65536
    X = torch.zeros(n, device="cuda")
    P = torch.empty(n, device="cuda")
    I = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mp_selfjoin_static(C.c_void_p(X.data_ptr()), n, 100, 25, C.c_void_p(P.data_ptr()),
                                C.c_void_p(I.data_ptr()), None)
    assert st == 1  # TSK_ERR_INVALID_ARG, nothing issued
