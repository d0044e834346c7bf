"""The C-ABI library builds, loads, and exports every entry point include/tsketch.h declares."""
import os
import re
import subprocess

import pytest

from paper_2311_03393_gb300 import _native, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsketch.h")


def _declared():
    src = open(HEADER).read()
    return re.findall(r"TSK_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def test_header_declares_the_five_entry_points():
    names = set(_declared())
    for fn in ("ts_sketch_build", "ts_sketch_update_dims", "mp_selfjoin", "discord_topk", "mp_backward"):
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    assert set(_native.exported_symbols()) == set(_declared())
    h = _native.lib()
    for name in _declared():
        assert hasattr(h, name)


def test_create_without_gpu_reports_an_error(libpath):
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = _native.lib().tsk_create(C.byref(h), 0, None)
    assert st != _native.TSK_OK and not h.value


def test_null_context_is_rejected(libpath):
    lib = _native.lib()
    assert lib.ts_sketch_build(None, None, 0, 0, None, 0, None, 0, 0, None, None) == 1
    assert lib.mp_selfjoin(None, None, 0, 0, None, None, 0, 0, 0, None, None) == 1


def test_dimension_detection_rejects_a_null_context(libpath):
    lib = _native.lib()
    assert lib.dimension_detection(None, None, 0, 0, None, 0, None, 0, 0, 0, 0, None, None, None, None, None,
                                   None, None, None, None, None) == 1



def _null_args(argtypes):
    """NULL for every pointer argument, 0 for every number."""
    import ctypes as C
    return [None if isinstance(a, type) and issubclass(a, (C._Pointer, C.c_void_p, C.c_char_p)) else 0
            for a in argtypes]


@pytest.mark.parametrize("name", sorted(n for n, (_, args) in _native.SIGNATURES.items()
                                        if args and args[0] is _native._P
                                        and n not in ("tsk_create", "tsk_destroy", "mp_selfjoin_static")))
def test_every_context_call_rejects_a_null_context(libpath, name):
    """Every entry point that takes a context returns TSK_ERR_INVALID_ARG for NULL (nothing
    launched); tsk_launch_count reports -1 and tsk_last_error says what was wrong."""
    lib = _native.lib()
    got = getattr(lib, name)(*_null_args(_native.SIGNATURES[name][1]))
    if name == "tsk_launch_count":
        assert got == -1
    elif name == "tsk_last_error":
        assert got == b"null context"
    else:
        assert _native.STATUS_NAMES.get(got) == "TSK_ERR_INVALID_ARG", (name, got)


@pytest.mark.parametrize("args", [
    dict(X=False, n=200, m=20, excl=5),              # no input
    dict(X=True, n=200, m=1, excl=5),                # m < 2
    dict(X=True, n=200, m=5000, excl=5),             # m > 4096
    dict(X=True, n=19, m=20, excl=5),                # n < m
    dict(X=True, n=200, m=20, excl=0),               # no exclusion zone
    dict(X=True, n=70000, m=20, excl=5),             # more windows than the static scratch holds
], ids=["null", "m1", "m_big", "n_small", "excl0", "too_long"])
def test_allocation_free_profile_rejects_bad_arguments_before_any_cuda_call(libpath, args):
    """mp_selfjoin_static checks its arguments before touching CUDA, so this runs without a GPU;
    the dummy device pointers are never dereferenced."""
    import ctypes as C
    lib = _native.lib()
    X = C.c_void_p(16) if args["X"] else None
    st = lib.mp_selfjoin_static(X, args["n"], args["m"], args["excl"], C.c_void_p(16), C.c_void_p(16), None)
    assert _native.STATUS_NAMES.get(st) == "TSK_ERR_INVALID_ARG"
