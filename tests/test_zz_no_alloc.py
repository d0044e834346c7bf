"""The allocation-free matrix-profile entry point (mp_selfjoin_static).

Some callers cannot allocate device memory (a monitor that must not allocate
after start-up, code inside another framework's memory pool or allocator
callback).  mp_selfjoin_static serves them from a fixed array in the library's
device memory.  Here it is called through the C ABI on two inputs in a row
and must agree with mp_selfjoin each time; the second call also checks that
the shared array's leftovers from the first call do not leak into its result.
This file is named to be collected last.
"""
import ctypes as C
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MP_REL_TOL = 1e-3


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
    floor = 1e-2 * math.sqrt(2 * m)
    for seed, n in ((300, 5000), (301, 2300)):
        x = np.cumsum(np.random.default_rng(seed).normal(size=n)).astype(np.float32)
        X = torch.from_numpy(x).cuda()
        P, I = _static_call(lib, X, n, m, excl)
        P_ref, I_ref = tsk.mp_selfjoin(X, [n], m, excl)
        torch.cuda.synchronize()
        l = n - m + 1
        P, I = P.cpu().numpy(), I.cpu().numpy()
        P_ref, I_ref = P_ref.cpu().numpy(), I_ref.cpu().numpy()
        assert np.all(np.isnan(P[l:])) and np.all(I[l:] == -1)
        err = np.abs(P[:l] - P_ref[:l]) / np.maximum(P_ref[:l], floor)
        assert err.max() <= MP_REL_TOL
        same = I[:l] == I_ref[:l]
        assert same.mean() > 0.999
        # where the neighbour differs it must be an equally near one
        assert np.all(np.abs(P[:l][~same] - P_ref[:l][~same]) <= MP_REL_TOL * np.maximum(P_ref[:l][~same], floor))


def test_static_entry_point_rejects_inputs_beyond_its_limit(libs):
    _, lib = libs
    n = 65536 + 100  # l = 65537 windows > 65536
    X = torch.zeros(n, device="cuda")
    P = torch.empty(n, device="cuda")
    I = torch.empty(n, dtype=torch.int32, device="cuda")
    st = lib.mp_selfjoin_static(C.c_void_p(X.data_ptr()), n, 100, 25, C.c_void_p(P.data_ptr()),
                                C.c_void_p(I.data_ptr()), None)
    assert st == 1  # TSK_ERR_INVALID_ARG, nothing issued
