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
